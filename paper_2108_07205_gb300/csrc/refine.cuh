// Algorithm 1 of the paper on the device: pre-computation for one local
// refinement (Sec. 3.1-3.4) and the Woodbury solve (Eq. wood).
#pragma once
#include "hbs.cuh"

namespace rw {

struct Wall {
  Curve curve;
  int n_panels = 0;
  Opts opts;
  Nodes nodes;  // original discretisation (panel order)
  Hbs hbs;      // A_oo at id_tol: inverse (direct solves, preconditioner) and forward
  Hbs hbs_op;   // A_oo forward at op_tol when that is tighter (else empty)
  // The forward representation used for residuals.
  const Hbs& op() const { return hbs_op.N ? hbs_op : hbs; }
  // Build hbs (with its FP32 and BF16 copies) and, when op_tol is tighter
  // than id_tol, hbs_op, on the wall's nodes.
  void build_hbs(cudaStream_t s);
};

// Side streams of one refinement: created by factor(), destroyed last (after
// every buffer allocated on them has been released).
struct SideStreams {
  cudaStream_t main = nullptr, s1 = nullptr, s2 = nullptr, s3 = nullptr;
  ~SideStreams();
};

// One added hole (App. B): x(t) = c + R (1 + a cos(k t)) (cos t, sin t),
// P panels equal in t.
struct HoleSpec {
  double cx, cy, R, a;
  int k, P;
};

// Recompression of one block of Q's low-rank factors (Sec. 3.4).  The
// blockwise IDs bound a block of Q through proxies that stand for every
// possible source or target near the modification, so their ranks can exceed
// the block's own.  A row ID of the skeleton block A(J, cols) (sketched when
// wide) gives A(J, cols) ~ T A(J[J'], cols), so L A(J, cols) ~ (L T)
// A(J[J'], cols): L (m x k, column major) takes the product and J the
// surviving skeleton rows; k shrinks to the new rank.  cols: the explicit
// column lists of an IdMatProb (n1/e1 in E1, n2/e2 in E2).
void recompress_rows(const NodesView& S, std::vector<int>& J, const IdMatProb& cols, const NodesView& E1, bool e1s,
                     const NodesView& E2, bool e2s, DBuf<double>& L, int m, int& k, double tol,
                     unsigned long long seed, cudaStream_t s);
// RW_RECOMPRESS=0 (diagnostics) keeps the blockwise ranks.
bool recompress_enabled();

// Runs a refinement program on bases 0, 1 (inputs), 3, 4 (outputs) and 5,
// with a stream-ordered workspace as base 2.
template <class T>
void run_prog(const GProgram<T>& P, const T* b0, const T* b1, T* b3, T* b4, T* b5, int nrhs, cudaStream_t s);

struct Refinement {
  SideStreams streams;  // first member: destroyed last
  const Wall* wall = nullptr;
  bool holes = false;                  // App. B: holes added, nothing cut
  std::vector<int> panels, levels;     // cut panels (window order) and levels
  int No = 0, Nk = 0, Nc = 0, Np = 0, Nn = 0;
  std::vector<int> Ic, Ik;             // point indices into the wall
  Nodes pn;                            // added nodes, window order
  Nodes nn;                            // refined nodes, refined order
  Hbs hpp;                             // A_pp (single leaf = dense inverse)
  bool pp_dense = false;
  int kf = 0, kn = 0, kpk = 0, kk = 0, k = 0;
  int kpk_id = 0;                      // rank of the A_pk ID(s) before recompression
  double cond_w = 0.0;                 // ||W||_1 ||W^-1||_1
  // factors: L_o (2No x kk), L_p (2Np x kpk); R blocks; X = A~^{-1} L; W^{-1}
  DBuf<double> Lo, Lp, Rkc, Rkp, Rpk, Xo, Xp, Winv;
  DBuf<int> dc;                  // c DOFs (2Nc) in o numbering
  DBuf<int> n_from_o, n_to_o;    // refined DOFs that are kept: (n index, o index)
  DBuf<int> n_from_p, n_to_p;    // refined DOFs that are added: (n index, p index)
  int nko = 0, nkp = 0;
  size_t bytes = 0;

  // The direct solve as one persistent program (bases: g, tau, workspace).
  Program solve_prog;
  mutable DBuf<double> solve_ws;
  void build_solve_program(cudaStream_t s);
  // Append this refinement's direct solve to a program: g = base gb + g_off
  // (ld ldg), tau = base tb + t_off (ld ldt), temporaries in base 2.
  void emit_solve(Program& P, int gb, long long g_off, int ldg, int tb, long long t_off, int ldt) const;
  // GEMV-program pieces of the batched iterative refinement, on ext-space
  // vectors (the o part at offset off, the p part at off + 2No, leading
  // dimension ld): g_n -> g_ext (zeros on I_c), the direct solve y =
  // A_ext^{-1} v (Algorithm 1), the operator y = (A~ + L R) x with the wall's
  // op_tol forward representation, and x_ext -> tau_n.  Workspace in base 2.
  void emit_to_ext(Program& P, int gb, long long g_off, int ldg, int eb, long long e_off, int lde) const;
  void emit_ext_direct(Program& P, int vb, long long vo, int ldv, int yb, long long yo, int ldy) const;
  void emit_ext_operator(Program& P, int xb, long long xo, int ldx, int yb, long long yo, int ldy) const;
  void emit_from_ext(Program& P, int eb, long long e_off, int lde, int tb, long long t_off, int ldt) const;
  // added (optional): the added nodes, 6 x N_p host array (x, y, nx, ny, w,
  // kappa) in window order; without it they are evaluated on the wall's curve
  void factor(const Wall& w, const std::vector<int>& panels, const std::vector<int>& levels, cudaStream_t s,
              const std::vector<double>* added = nullptr);
  // App. B: holes added inside the wall (no point cut).  The system is
  // [A_kk A_kp; A_pk A_pp] with A_pp = 1/2 I + D + S on the holes (dense,
  // singular rule), A_kp the holes' combined field on the wall and A_pk the
  // wall's double layer on the holes; Q = [0 A_kp; A_pk 0] ~ L R.
  void factor_holes(const Wall& w, const std::vector<HoleSpec>& holes, cudaStream_t s);
  // y = A_nn x, the exact refined (or holed) operator, entries on the fly
  // (the dense hole block from its stored matrix).  x, y: 2Nn x nrhs.
  void apply_nn(const double* x, double* y, int nrhs, cudaStream_t s) const;
  // Velocity / pressure of a density tau (2Nn x nrhs) at targets (2 x nt).
  void velocity(const double* tau, int nrhs, int nt, const double* targets, double* u, cudaStream_t s) const;
  void pressure(const double* tau, int nrhs, int nt, const double* targets, double* p, cudaStream_t s) const;
  // Direct solve, device buffers: g, tau (2Nn x nrhs): one persistent launch
  // per 8 right-hand sides.  solve_direct_levels is the same computation as
  // a sequence of per-level launches.
  void solve_direct(const double* g, double* tau, int nrhs, cudaStream_t s) const;
  void solve_direct_levels(const double* g, double* tau, int nrhs, cudaStream_t s) const;
  // Direct solve followed by `steps` rounds of iterative refinement against
  // the exact refined operator (on-the-fly N-body evaluation of A_nn).
  void solve_refined(const double* g, double* tau, int nrhs, int steps, cudaStream_t s) const;
  // Woodbury apply in ext space: (yo, yp) <- Ainv_ext (yo, yp), yo/yp hold
  // A~^{-1} g on entry (ld 2No / 2Np).
  void woodbury_correct(double* yo, double* yp, int nrhs, cudaStream_t s) const;
  // FGMRES on A~ + L R with the Woodbury preconditioner, its HBS sweeps in
  // FP32 (or with BF16 matrices when bf16 is set).  mixed: the operator's
  // products in double-FP32 and the preconditioner's Woodbury correction in
  // FP32 (W^{-1} in FP64), for nrhs > 8 (RW_MODE_GMRES_MIXED).
  void solve_gmres(const double* g, double* tau, int nrhs, cudaStream_t s, int* iters, double* relres,
                   bool bf16 = false, bool mixed = false) const;
  // ext-space operator y = (A~ + L R) x (FP64)
  void apply_els(const double* xo, const double* xp, double* yo, double* yp, int nrhs, cudaStream_t s) const;
  // the same with every product in double-FP32 (FP64-level accuracy)
  void apply_els_df(const double* xo, const double* xp, double* yo, double* yp, int nrhs, cudaStream_t s) const;
  // Algorithm 1 solve plus iterative refinement against apply_els until the
  // relative residual is <= gmres_tol: FP64 (RW_MODE_DIRECT_IR), or with
  // every product of the solves and of the operator in double-FP32 when df
  // is set (RW_MODE_DIRECT_IR_DF).
  void solve_ir(const double* g, double* tau, int nrhs, cudaStream_t s, int* iters, double* relres,
                bool df = false) const;
  // Many right-hand sides: the whole ELS operator, the whole FP64 direct
  // solve (Algorithm 1 in ext space) and the low-precision preconditioner as
  // GEMM programs, the wall's and the refined arc's trees side by side in
  // the same phases with the Woodbury terms (built on first use).
  // ELS operator: bases 0 = x_o, 1 = x_p, 2 = workspace, 3 = y_o, 4 = y_p.
  const GProgram<double>& els_prog(bool df, cudaStream_t s) const;
  // The same operator with FP32 factors and vectors (the relaxed FGMRES
  // iterations of the mixed mode): same bases, FP32.
  const GProgram<float>& els_prog32(cudaStream_t s) const;
  // Direct solve in ext space: bases 0 = g_o, 1 = g_p, 2 = workspace,
  // 3 = y_o, 4 = y_p; FP64 factors, or their double-FP32 copies (df).
  const GProgram<double>& dir_prog(cudaStream_t s, bool df = false) const;
  // Preconditioner, FP32 vectors: part a = sweeps and r = R y (bases 0 = v_o,
  // 1 = v_p, 2 = workspace, 3 = y_o, 4 = y_p, 5 = r, k x nrhs); part b =
  // y -= X z (bases 3, 4, and 5 = z); W^{-1} is applied in FP64 between them.
  const GProgram<float>& pre_prog_a(bool bf16, cudaStream_t s) const;
  const GProgram<float>& pre_prog_b(cudaStream_t s) const;
  mutable GProgram<double> g_els64, g_elsdf, g_dir64, g_dirdf;
  mutable GProgram<float> g_pre32, g_pre16, g_preb, g_els32;
  // double-FP32 copies of L, R, X and W^{-1}, FP32 copies of R, X and L
  // (made on first use)
  void make_mixed() const;
  mutable bool has_mixed = false;
  mutable DBuf<float2> Lo2, Lp2, Rkc2, Rkp2, Rpk2, Xo2, Xp2, Winv2;
  mutable DBuf<float> Rkc32, Rkp32, Rpk32, Xo32, Xp32, Lo32, Lp32;
  ~Refinement();

 private:
  // X = H^{-1} L (m x k): FP64 sweeps, or FP32 (opts.mixed_factor 1) or
  // double-FP32 (2) sweeps
  void solve_x(const Hbs& H, const double* L, double* X, int m, int k, cudaStream_t s) const;
  // a6 and the solve program, shared by both factorisations: W = I + R X,
  // W^{-1}, its condition estimate, and the persistent solve program.
  void form_w(cudaStream_t s);
};

}  // namespace rw
