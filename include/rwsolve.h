/*
 * rwsolve -- refined-wall Stokes solver for GB300 (sm_103a).
 *
 * Fast direct solve of the interior Stokes double-layer boundary integral
 * equation on a locally refined wall, after Zhang, Gillman and Veerapaneni,
 * "A fast direct solver for integral equations on locally refined boundary
 * discretizations" (arXiv 2108.07205):
 *
 *   A = -1/2 I + D + N                      (Sec. 2, Eq. interior_BIE_discretized2)
 *   A_ext = A~ + Q,  A~ = blkdiag(A_oo, A_pp)   (Sec. 3.2, Eq. extendedlLinearSystem)
 *   tau_ext = A~^{-1} g - A~^{-1} L (I + R A~^{-1} L)^{-1} R A~^{-1} g   (Eq. wood)
 *
 * with A_oo^{-1} a hierarchically block separable (HBS) compressed inverse of
 * the reference wall built once (rw_hbs_build), Q ~= L R the uniform row-ID
 * factorisation of Sec. 3.3-3.4 built per refinement (rw_refine_factor), and
 * Algorithm 1's solve (rw_solve).
 *
 * Conventions (all calls):
 *  - mu = 1; r = x - y; degrees of freedom interleaved (x, y) per point.
 *  - FP64 arrays; column-major with leading dimension = number of rows.
 *  - Pointers marked "host or device" are classified with
 *    cudaPointerGetAttributes; host buffers are copied in and out inside the
 *    call on the given stream and the call returns after the copy back.
 *  - The library owns every handle and all device memory behind it.  The
 *    caller owns the buffers it passes.
 *  - Calls are ordered on the CUDA stream passed as `stream` (a cudaStream_t;
 *    NULL means the legacy default stream).  Handles are not thread safe.
 *  - Return value: RW_OK (0) or a negative RW_ERR_* code.  rw_last_error()
 *    returns a thread-local message for the last failure on this thread.
 */
#ifndef RWSOLVE_H
#define RWSOLVE_H

#ifdef __cplusplus
extern "C" {
#endif

#define RW_OK 0
#define RW_ERR_INVALID (-1)        /* bad argument, shape or handle            */
#define RW_ERR_OOM (-2)            /* device allocation or admission refused   */
#define RW_ERR_SINGULAR (-3)       /* pivot below threshold (W, A_pp, D~)       */
#define RW_ERR_NOT_CONVERGED (-4)  /* GMRES stopped at maxit above tolerance    */
#define RW_ERR_TIMEOUT (-5)        /* a bounded device wait gave up             */
#define RW_ERR_CUDA (-6)           /* CUDA runtime error                        */

/* Built-in wall curves, t in [0, 2 pi), counter-clockwise.
 *  RW_CURVE_STAR:    x(t) = s (1 + a cos(k t)) (cos t, sin t);
 *                    params = {a, k, s}.
 *  RW_CURVE_CHANNEL: superellipse (A cos t, B sin t) (cos^p t + sin^p t)^(-1/p)
 *                    with y scaled by 1 - delta (1 + cos(pi x / A)) / 2;
 *                    params = {A, B, p, delta}.  The synthetic stand-in for
 *                    the paper's spline channel (Sec. 5.1). */
#define RW_CURVE_STAR 0
#define RW_CURVE_CHANNEL 1
#define RW_CURVE_NODES 2   /* wall given by explicit nodes (rw_hbs_build_nodes) */

typedef struct {
  int curve_kind;     /* RW_CURVE_*                                          */
  int n_panels;       /* P equal panels in t, 16 Gauss-Legendre points each   */
  double params[8];   /* curve parameters, see above                        */
} rw_wall_desc;

typedef struct {
  int leaf_points;          /* HBS leaf size in points (default 64)          */
  double id_tol;            /* ID tolerance eps of Def. 3.1 (default 1e-12)  */
  int n_proxy;              /* points on an HBS proxy circle (default 64)    */
  double proxy_ratio;       /* HBS proxy radius / node radius (default 2.0)  */
  int n_proxy_refine;       /* points on P^div and P^bas (default 96)        */
  double div_ratio;         /* P^div radius / radius of Gamma_r (default 2)  */
  double bas_ratio;         /* P^bas radius / radius of Gamma_r (default 1.5)*/
  int dense_pp_max_points;  /* A_pp inverted densely up to this many added
                               points, else by an HBS of the refined arc
                               (Alg. 1 step 2; default = leaf_points)         */
  int sketch_cols;          /* ID matrices wider than this are compressed by
                               a random +-1 sketch first (default 2048)       */
  double gmres_tol;         /* relative residual target (default 1e-10)      */
  int gmres_maxit;          /* iterations per restart cycle (default 30)     */
  int gmres_restarts;       /* restart cycles (default 4)                    */
  unsigned long long seed;  /* seed of the sketch generator                  */
  double hole_div_ratio;    /* P^div radius / radius of an added hole (App. B;
                               default 4: the wall points inside are taken
                               explicitly, so a wider circle lowers the
                               A_pk rank toward the block's own)            */
  double op_tol;            /* tolerance of the operator representation that
                               residuals are computed with (FGMRES, iterative
                               refinement; Sec. 4.2); 0 (default) = id_tol.
                               When smaller than id_tol, rw_hbs_build keeps a
                               second forward HBS of A_oo at op_tol beside the
                               inverse at id_tol, and rw_refine_factor /
                               rw_holes_factor compute the row IDs of Q and
                               the representation of A_pp at op_tol, so that
                               A~ + L R matches A_ext to about op_tol while the
                               reference wall's inverse stays at id_tol      */
  int mixed_factor;         /* 0 (default): refinements of this wall compute
                               X = A~^{-1} L with FP64 sweeps.  1: with FP32
                               sweeps, 2: with double-FP32 sweeps; W = I +
                               R X is formed from X in FP64 either way.
                               Such a factorisation serves only the
                               iterative modes (RW_MODE_GMRES_*,
                               RW_MODE_DIRECT_IR, RW_MODE_DIRECT_IR_DF; with
                               1 they need more iterations);
                               RW_MODE_DIRECT, RW_MODE_DIRECT_REFINED and
                               batches refuse it with RW_ERR_INVALID        */
} rw_opts;

typedef struct {
  int n_points;        /* N on the wall                                      */
  int levels;          /* tree depth (root = 0, leaves = levels)             */
  int max_rank;        /* largest node rank                                  */
  long long inv_elems; /* matrix entries read by one inverse sweep           */
  long long fwd_elems; /* matrix entries read by one forward apply           */
  long long bytes;     /* device bytes held by the handle                    */
  long long op_fwd_elems; /* entries read by one forward apply of the operator
                          representation (= fwd_elems unless op_tol < id_tol) */
} rw_hbs_stats;

typedef struct {
  int n_k, n_c, n_p;   /* points kept, cut and added (Sec. 3.1)              */
  int n_n, n_ext;      /* N_n = N_k + N_p, N_ext = N_k + N_c + N_p           */
  int k_far, k_near, k_pk;  /* ranks of the far, near and A_pk row IDs       */
  int k;               /* Woodbury size k <= k_far + k_near + k_pk after the
                          recompression of Sec. 3.4 (row IDs of the skeleton
                          blocks of R)                                       */
  int pp_dense;        /* 1 if A_pp was inverted densely                     */
  int pp_levels;       /* tree depth of the refined-arc HBS (0 if dense)     */
  long long bytes;     /* device bytes held by the handle                    */
} rw_ref_stats;

typedef struct {
  int iters;             /* GMRES iterations (0 for the direct path)         */
  double rel_residual;   /* GMRES: final relative residual of the ELS        */
  int k_woodbury;        /* Woodbury size k of the refinement                */
  double cond_w;         /* 1-norm condition estimate of W = I + R X:
                            ||W||_1 ||W^-1||_1 (computed at factorisation)   */
} rw_info;

/* A wall given by explicit nodes: n = 16 P points in panel order (P panels of
 * 16 Gauss-Legendre points, counter-clockwise), with unit outward normals
 * (nx, ny), quadrature weights w (Gauss-Legendre weight times |x'(t)| times
 * the panel's half-width in t) and signed curvature kappa.  Each array holds
 * n values, host or device. */
typedef struct {
  int n;
  const double *x, *y, *nx, *ny, *w, *kappa;
} rw_nodes;

typedef struct rw_hbs_s* rw_hbs_t;   /* reference wall: HBS forward + inverse */
typedef struct rw_ref_s* rw_ref_t;   /* one refinement: Woodbury factors       */

/* Fill *o with the defaults listed above. */
int rw_default_opts(rw_opts* o);

/* a0. Build the reference wall's nodes, the proxy-compressed HBS
 * representation of A_oo and its HBS inverse (Sec. 3 preamble and Sec. 4.2:
 * the fast direct solver for the original discretisation is taken as given;
 * the HBS construction and inversion follow Gillman-Young-Martinsson 2012).
 * opts may be NULL (defaults).  On success *out owns all device memory. */
int rw_hbs_build(const rw_wall_desc* wall, const rw_opts* opts, void* stream,
                 rw_hbs_t* out);

/* a0 for the exterior problem (Sec. 2.2, Fig. demo_figs (b)): the fluid
 * fills the plane outside the closed curve (RW_CURVE_STAR or
 * RW_CURVE_CHANNEL, n_panels >= 8 equal panels in t), the velocity is the
 * combined field u = (D + S) tau and the density solves
 * 1/2 tau + (D + S) tau = g (Eq. exterior_BIE; full rank, no N term).  The
 * single layer's logarithm takes Legendre product integration (the
 * generalised Gaussian corrections of Sec. 5, exact for the density's
 * degree-15 interpolant on a panel, geometry exact) wherever a target lies
 * within 2 half-widths (in t) of the source panel's midpoint; the plain
 * panel rule elsewhere.  Every later call takes the handle as for an
 * interior wall (Sec. 3 applies to exterior problems unchanged: the Remark
 * closing Sec. 3.1): rw_refine_factor (nodes of the sub-panels evaluated on
 * the curve; rw_refine_factor_nodes is refused), rw_solve in every mode,
 * rw_apply_refined, velocity (D + S, plain rule: targets away from the
 * curve), pressure, batches and the server.  rw_holes_factor and rw_hbs_save
 * refuse an exterior wall with RW_ERR_INVALID. */
int rw_hbs_build_exterior(const rw_wall_desc* wall, const rw_opts* opts, void* stream, rw_hbs_t* out);

/* a0 for a wall given by its nodes (any geometry: the paper's spline
 * channel, fish or tube discretised elsewhere).  Checks n = 16 P >= 16,
 * finite values, positive weights and unit normals (|n| within 1e-8 of 1),
 * else RW_ERR_INVALID.  Such a wall has no curve: refine it with
 * rw_refine_factor_nodes. */
int rw_hbs_build_nodes(const rw_nodes* nodes, const rw_opts* opts, void* stream, rw_hbs_t* out);

/* Checkpoint and restore of a built wall (nodes, curve, options, HBS
 * forward and inverse factors) in a binary file, little-endian, for the same
 * library version; a restored handle gives the same results as the one saved.
 * Load allocates on the current device.  Errors: RW_ERR_INVALID for an
 * unreadable, truncated or foreign file. */
int rw_hbs_save(rw_hbs_t h, const char* path);
int rw_hbs_load(const char* path, void* stream, rw_hbs_t* out);

int rw_hbs_stats_get(rw_hbs_t h, rw_hbs_stats* s);

/* Copy the wall's nodes into `out` (host or device, 6 x N column-major:
 * x, y, nx, ny, w, kappa per point, panel order). */
int rw_hbs_nodes(rw_hbs_t h, double* out, void* stream);

/* x = A_oo^{-1} b on the reference wall by the HBS inverse sweep.
 * b, x: 2N x nrhs (host or device; may not alias). */
int rw_hbs_apply_inverse(rw_hbs_t h, int nrhs, const double* b, double* x,
                         void* stream);

/* Allocation-free x = A_oo^{-1} b (no counterpart in the paper: a library
 * service).  For callers that cannot let the library allocate or free device
 * memory during a solve -- e.g. a host application whose device memory is
 * owned by another framework's pool, or a latency-critical loop where an
 * allocation or free could synchronise the device.  Same result as
 * rw_hbs_apply_inverse; every temporary comes from one fixed 32 MiB device
 * array inside the library (held by every GPU that loads the library until
 * exit), so b and x must be device pointers and nrhs is limited to 1..8;
 * larger problems return RW_ERR_INVALID with a message.  The first call on a
 * device resolves the array's address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the array and it keeps the last call's contents (the sweep writes every
 * entry before reading it); calls that overlap on the GPU race on it, so
 * order them on one stream. */
int rw_hbs_apply_inverse_noalloc(rw_hbs_t h, int nrhs, const double* b,
                                 double* x, void* stream);

/* y = A_oo x by the HBS forward representation (used for GMRES mat-vecs). */
int rw_hbs_apply_forward(rw_hbs_t h, int nrhs, const double* x, double* y,
                         void* stream);

/* a1-a6. Algorithm 1 pre-computation for one local refinement (Sec. 3.1-3.4):
 * cut the n_cut panels panel_ids[] and replace panel_ids[i] by 2^levels[i]
 * equal sub-panels; build the added nodes, A_pp^{-1}, the row-ID factors
 * Q ~= L R, X = A~^{-1} L and the LU factors of W = I + R X.  panel_ids is one
 * or more regions, each a contiguous run of panels modulo P given in window
 * order (consecutive entries i, i+1 with panel_ids[i+1] = panel_ids[i] + 1 mod
 * P belong to one region), at most 8 regions: several refined regions grouped
 * in one refinement share one factorisation of Q (Sec. 5.3, the Remark on
 * grouping two refined regions, e.g. those of two consecutive time steps);
 * each region gets its own proxy circles.  panel_ids and levels are host
 * arrays; panels must be distinct, levels in 0..12.
 * The handle borrows h, which must outlive it.  Its device memory is
 * allocated in stream order on `stream`, which must stay valid until
 * rw_ref_free. */
int rw_refine_factor(rw_hbs_t h, int n_cut, const int* panel_ids,
                     const int* levels, void* stream, rw_ref_t* out);

/* As rw_refine_factor with the added nodes given by the caller (any wall,
 * required for walls built from nodes): added holds the 16 x 2^levels[i]
 * nodes of each cut panel's sub-panels, cut panels in window order, points
 * in parameter order within each (same checks as rw_hbs_build_nodes). */
int rw_refine_factor_nodes(rw_hbs_t h, int n_cut, const int* panel_ids, const int* levels,
                           const rw_nodes* added, void* stream, rw_ref_t* out);

/* One hole added inside the wall (App. B): the closed curve
 * x(t) = (cx, cy) + radius (1 + a cos(k t)) (cos t, sin t), t in [0, 2 pi),
 * counter-clockwise, cut into n_panels panels equal in t with 16
 * Gauss-Legendre points each (the paper's holes are circles, a = 0, with 10
 * panels, Sec. 5.2).  Requirements: radius > 0, 0 <= a < 1, 0 <= k <= 64,
 * 5 <= n_panels <= 256; the holes lie inside the wall's fluid region, apart
 * from the wall and from one another (the library checks only that the
 * holes' enclosing circles do not overlap). */
typedef struct {
  double cx, cy, radius, a;
  int k;
  int n_panels;
} rw_hole;

/* App. B (Eq. simple_ext) with the combined-field BIE of Eq. exterior_BIE on
 * the holes: factor the wall with n_holes (1..8, at most 1024 hole points
 * in all) holes added, nothing cut.  Unknowns: the wall's points (panel
 * order) then the holes' points (hole by hole, panel by panel), interleaved
 * (x, y) per point; N_c = 0, N_p = hole points.  The system is
 *   [A_kk  A_kp] with A_kk = -1/2 I + D + N (the wall operator, N on the
 *   [A_pk  A_pp]      wall only), A_pp = 1/2 I + D + S on the holes
 * (log-singular single layer by product integration of the density's
 * interpolant on each target's own panel and two panels on either side), A_kp = the holes' combined field w_j (D + S) on
 * the wall, A_pk = the wall's double layer w_j D on the holes.  The velocity
 * (rw_solve targets) is the wall's double layer plus the holes' combined
 * field; rw_pressure likewise.  The returned handle works with every rw_ref_t
 * call (rw_solve in all modes, rw_apply_refined, rw_stokeslet_data,
 * rw_pressure, rw_ref_nodes, batches); it borrows the wall, which must
 * outlive it.  Errors: RW_ERR_INVALID (arguments, overlapping holes),
 * RW_ERR_SINGULAR (A_pp or W not invertible), RW_ERR_OOM, RW_ERR_CUDA. */
int rw_holes_factor(rw_hbs_t wall, int n_holes, const rw_hole* holes, void* stream, rw_ref_t* out);

int rw_ref_stats_get(rw_ref_t r, rw_ref_stats* s);

/* Copy the refined nodes in refined order (6 x N_n, as rw_hbs_nodes). */
int rw_ref_nodes(rw_ref_t r, double* out, void* stream);

/* Boundary data from point forces (Eq. stokeslet): g(x_i) = sum_s S(x_i, y_s) f_s
 * at the refined nodes.  src: 2 x n_src (x, y); f: 2 x n_src x nrhs;
 * g: 2 N_n x nrhs.  All host or device. */
int rw_stokeslet_data(rw_ref_t r, int n_src, const double* src, int nrhs,
                      const double* f, double* g, void* stream);

#define RW_MODE_DIRECT 0      /* Algorithm 1 solve, FP64                     */
#define RW_MODE_GMRES_FP32 1  /* FGMRES (FP64) on A~ + L R, preconditioned by
                                 Algorithm 1 with FP32 HBS sweeps (Sec. 4.2) */
#define RW_MODE_DIRECT_REFINED 2  /* Algorithm 1 solve plus one step of
                                 iterative refinement against the exact
                                 refined operator A_nn (on-the-fly N-body
                                 evaluation); removes the compression error
                                 amplified by the conditioning of A_nn      */
#define RW_MODE_GMRES_BF16 3  /* as RW_MODE_GMRES_FP32 with the HBS sweeps'
                                 matrices in BF16 (FP32 vectors and
                                 accumulation, Sec. 4.2): converges on
                                 well-conditioned walls in more iterations;
                                 RW_ERR_NOT_CONVERGED where the BF16 rounding
                                 times the conditioning of A_oo exceeds one */
#define RW_MODE_DIRECT_IR 4   /* the plain FP64 path to a certified residual:
                                 Algorithm 1 solve, then FP64 iterative
                                 refinement tau += A_ext^{-1} (g - (A~ + L R)
                                 tau) with the operator in its op_tol
                                 representation, until the relative residual
                                 is <= gmres_tol (at most gmres_maxit
                                 corrections; iters = corrections made) */
#define RW_MODE_GMRES_MIXED 5 /* as RW_MODE_GMRES_FP32, with the operator's
                                 products for nrhs > 8 in double-FP32: every
                                 FP64 factor of A~ + L R is held as a pair of
                                 FP32 numbers (hi + lo) and each product and
                                 sum is compensated (exact FMA product error,
                                 two-sum accumulation, FP64 every 128 terms),
                                 so the residual keeps FP64-level accuracy
                                 (relative error ~1e-14 per product) from the
                                 FP32 units; Krylov vectors, Hessenberg
                                 matrix, X and W^{-1} stay FP64 */
#define RW_MODE_DIRECT_IR_DF 6 /* RW_MODE_DIRECT_IR with every product in
                                 double-FP32 (the representation above): the
                                 HBS inverse sweeps of A_oo and A_pp, the
                                 Woodbury terms R, W^{-1} and X of Algorithm
                                 1 and the op_tol operator A~ + L R of the
                                 corrections; vectors, sums of corrections
                                 and residual norms stay FP64.  One direct
                                 solve reaches a relative residual near
                                 1e-14 x the conditioning of A_nn, each
                                 correction multiplies it by about as much  */

/* y = A_nn tau with every entry of the refined operator evaluated on the fly
 * (Sec. 2, Eq. interior_BIE_discretized2 on the refined nodes): the exact
 * residual of any solve.  tau, y: 2 N_n x nrhs (host or device, no alias). */
int rw_apply_refined(rw_ref_t r, int nrhs, const double* tau, double* y,
                     void* stream);

/* s1-s3 (and m1). Solve the refined system for nrhs right-hand sides:
 * g: 2 N_n x nrhs boundary data in refined order; tau: 2 N_n x nrhs density
 * (output, refined order); if n_targets > 0, u: 2 n_targets x nrhs interior
 * velocity u(x) = sum_j w_j D(x, y_j) tau_j at targets (2 x n_targets).
 * info may be NULL (iters = GMRES iterations, or 1 for the refined direct
 * mode; rel_residual = final GMRES relative residual of the ELS; k_woodbury
 * and cond_w describe the refinement's Woodbury operator). */
int rw_solve(rw_ref_t r, int nrhs, const double* g, double* tau, int n_targets,
             const double* targets, double* u, int mode, void* stream,
             rw_info* info);

/* Interior pressure matching the double-layer velocity (Sec. 2):
 * p(x) = sum_j w_j P(x, y_j) . tau_j with P_j(x, y) = (1/pi)(-n_j(y) / r^2 +
 * 2 r_j (r . n(y)) / r^4), mu = 1, for a refined density tau (2 N_n x nrhs,
 * refined order) at targets (2 x n_targets); p: n_targets x nrhs.  The
 * pressure of an interior flow is fixed up to a constant; this is the
 * representation's.  All host or device. */
int rw_pressure(rw_ref_t r, int nrhs, const double* tau, int n_targets, const double* targets, double* p,
                void* stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (diagnostics: benchmarks difference it around a timed region). */
unsigned long long rw_kernel_launches(void);

/* Serving loop (the paper has no serving layer):
 * continuous batching of refined-wall solve requests against resident walls.
 * rw_server_create starts n_workers host threads, each with its own CUDA
 * stream on the current device; requests queue FIFO and are admitted while
 * the estimated device memory of the admitted requests stays within
 * max_device_bytes (a request is always admitted when nothing else runs), so
 * requests arriving while others run start as memory frees up and their
 * kernels overlap on the device.  A request runs rw_refine_factor, boundary
 * data from point forces (rw_stokeslet_data), rw_solve and the velocity at
 * targets, and copies tau (2 N_n x nrhs) and u (2 n_targets x nrhs) to the
 * caller's host buffers, which must stay valid until the request completes.
 * Inputs are copied at submission.  Each result depends only on its own
 * request.  rw_server_wait blocks and returns the request's status;
 * rw_server_destroy finishes every queued request first. */
typedef struct rw_server_s* rw_server_t;
typedef struct {
  rw_hbs_t wall;
  int n_cut;
  const int* panel_ids;   /* host, n_cut (as rw_refine_factor)              */
  const int* levels;      /* host, n_cut                                    */
  int nrhs;
  int n_src;
  const double* src;      /* host, 2 x n_src                                */
  const double* f;        /* host, 2 x n_src x nrhs                         */
  int n_targets;
  const double* targets;  /* host, 2 x n_targets (may be NULL if none)      */
  double* tau;            /* host output, 2 N_n x nrhs                      */
  double* u;              /* host output, 2 n_targets x nrhs (or NULL)      */
  int mode;               /* RW_MODE_*                                      */
} rw_request;
int rw_server_create(int n_workers, long long max_device_bytes, rw_server_t* out);
int rw_server_submit(rw_server_t s, const rw_request* req, long long* ticket);
/* status: 1 queued or running, 0 done, < 0 the request's error code. */
int rw_server_poll(rw_server_t s, long long ticket, int* status, double* latency_ms);
int rw_server_wait(rw_server_t s, long long ticket, double* latency_ms);
/* Factor reuse across requests: keep each request's refinement
 * pre-computation (a1-a6) after it completes, up to max_bytes of device
 * memory counted in the server's budget, keyed by (wall, panel_ids, levels);
 * a request with the same key skips rw_refine_factor's work.  Least recently
 * used entries are evicted beyond max_bytes or when a waiting request needs
 * the memory.  0 (the default) disables the cache and frees its unused
 * entries.  With a cache, walls must outlive the server. */
int rw_server_set_cache(rw_server_t s, long long max_bytes);
/* Cache hits and misses so far and the device bytes the cache holds. */
int rw_server_stats(rw_server_t s, long long* hits, long long* misses, long long* cache_bytes);
int rw_server_destroy(rw_server_t s);

/* Batched solve of many refined walls (the paper
 * solves one wall at a time): the direct solves (Algorithm 1, s1-s3) of n
 * refinements, each on its own wall, run as one persistent cooperative launch
 * per 8 right-hand sides with phases aligned across the instances.  The
 * refinements must outlive the batch.  Right-hand sides of all instances are
 * stacked: g and tau are G x nrhs column-major (host or device), where
 * instance i occupies rows offsets[i] .. offsets[i+1]-1 (rw_batch_rows fills
 * offsets[0..n], offsets[n] = G) in its refined order.  use_graph != 0
 * captures the launch in a CUDA graph on first use per nrhs and replays it.
 * rw_batch_autotune times GEMV tiles of 16, 32 and 64 rows on the batch and
 * keeps the fastest (appended to the file named by RW_AUTOTUNE_CACHE, if set,
 * and read back by later batches of the same shape). */
typedef struct rw_batch_s* rw_batch_t;
int rw_batch_create(int n, const rw_ref_t* refs, void* stream, rw_batch_t* out);
int rw_batch_rows(rw_batch_t b, long long* offsets);
int rw_batch_autotune(rw_batch_t b, int nrhs, void* stream, int* tile_rows, float* ms);
int rw_batch_solve(rw_batch_t b, int nrhs, const double* g, double* tau, int use_graph, void* stream);
/* The batch solved to a certified residual (Sec. 4.2, as RW_MODE_DIRECT_IR
 * for each instance): Algorithm 1 for every instance in one persistent
 * launch per 8 right-hand sides, then FP64 corrections tau_ext +=
 * A_ext^{-1} (g_ext - (A~ + L R) tau_ext), every instance's operator (its
 * wall's op_tol forward HBS, A_pp and L R) applied in one launch per 8
 * right-hand sides, until the worst relative residual over all instances and
 * right-hand sides is <= tol, at most maxit corrections.  iters and relres
 * (may be NULL) receive the corrections made and that worst residual;
 * RW_ERR_NOT_CONVERGED if it stayed above tol.  Same g/tau layout as
 * rw_batch_solve; also takes refinements whose X is not FP64
 * (opts.mixed_factor), which rw_batch_solve refuses. */
int rw_batch_solve_ir(rw_batch_t b, int nrhs, const double* g, double* tau, double tol, int maxit, void* stream,
                      int* iters, double* relres);
void rw_batch_free(rw_batch_t b);

/* Opt-in kernel profiler (diagnostics, no counterpart in the paper).
 * rw_profile(1) clears the records and starts recording a pair of CUDA events
 * around every kernel launch of this library, on the stream of that launch,
 * with the launch's algorithmic flops and bytes (GEMM 2mnk, GEMV 2mn*nrhs,
 * Gauss-Jordan 2n^3, column-pivoted QR 4 flops per trailing entry per pivot
 * step, counted on the device).  rw_profile(0) stops.  rw_profile_read
 * synchronises the device and fills out[RW_KCLASS_COUNT] with per-class
 * launch counts, summed event durations (ms), flops and bytes. */
#define RW_KCLASS_ID 0       /* column-pivoted QR / interpolative decomposition */
#define RW_KCLASS_GEMM 1     /* batched tiled GEMM (FP64)                        */
#define RW_KCLASS_GEMV 2     /* batched GEMV: the HBS sweeps and Woodbury apply  */
#define RW_KCLASS_INVERSE 3  /* batched Gauss-Jordan inverse                     */
#define RW_KCLASS_EVAL 4     /* kernel-entry, proxy, node and N-body evaluation  */
#define RW_KCLASS_OTHER 5    /* copies, gathers, ID bookkeeping                  */
#define RW_KCLASS_GEMM_F32 6 /* batched GEMM with FP32 accumulation (FP32 or BF16
                                matrices): low-precision sweeps, many RHS       */
#define RW_KCLASS_GEMM_DF 7  /* double-FP32 GEMM: FP64-accurate operator
                                products of RW_MODE_GMRES_MIXED                 */
#define RW_KCLASS_COUNT 8
typedef struct {
  long long launches;
  double ms;
  double flops;
  double bytes;
} rw_kernel_stat;
int rw_profile(int enable);
int rw_profile_read(rw_kernel_stat* out, int n);

void rw_ref_free(rw_ref_t r);
void rw_hbs_free(rw_hbs_t h);
const char* rw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RWSOLVE_H */
