// Hierarchically block separable (HBS) representation of A on a node set and
// its inverse, after Gillman, Young and Martinsson (2012), which the paper
// takes as its fast direct solver for the original discretisation (Sec. 3
// preamble, Sec. 4.2).  Also the interpolative-decomposition helpers shared
// with the refinement factorisation.
#pragma once
#include <memory>
#include "dense.cuh"
#include "eval.cuh"
#include "program.cuh"
#include "gprogram.cuh"

namespace rw {

struct Opts {
  int leaf_points = 64;
  double id_tol = 1e-12;
  int n_proxy = 64;
  double proxy_ratio = 2.0;
  int n_proxy_refine = 96;
  double div_ratio = 2.0;
  double bas_ratio = 1.5;
  int dense_pp_max_points = 64;
  int sketch_cols = 2048;
  int sketch_width = 192;
  double gmres_tol = 1e-10;
  int gmres_maxit = 30;
  int gmres_restarts = 4;
  unsigned long long seed = 0x5eed2108ull;
  double hole_div_ratio = 4.0;
  // Tolerance of the operator used for residuals (FGMRES and iterative
  // refinement); 0: the same as id_tol.  When tighter, the wall keeps a
  // second forward representation at op_tol and a refinement's IDs and A_pp
  // are computed at op_tol.
  double op_tol = 0.0;
  // How refinements compute X = A~^{-1} L (a factorisation for the iterative
  // modes only when set; see rw_opts.mixed_factor): 0 FP64 sweeps, 1 FP32
  // sweeps, 2 double-FP32 sweeps
  int mixed_factor = 0;
  double factor_tol() const { return (op_tol > 0.0 && op_tol < id_tol) ? op_tol : id_tol; }
};

// A list of row-interpolative decompositions evaluated on the fly: each job
// is an IdMatProb (without output) whose matrix is optionally compressed by a
// +-1 sketch when it has more than `sketch_cols` columns.
class IdBatch {
 public:
  struct Job {
    IdMatProb spec;
    int sk_width = 0;  // 0: no sketch; else rows of the sketched W
    int nr = 0;        // rows of W handed to the QR
    size_t woff = 0, moff = 0, noff = 0;
  };
  std::vector<Job> jobs;
  DBuf<double> W, norms;
  DBuf<int> piv, rank;
  std::vector<int> h_rank;
  // Jobs 2i and 2i+1 are a node's row and column IDs: a run over all jobs
  // factors each pair with a joint stopping rule (both at the larger rank).
  bool paired = false;

  int add(const IdMatProb& spec, int sketch_cols, int sketch_width);
  // Evaluate (all jobs, or the listed subset) and factor.  min_rank/max_rank
  // are per job (empty: 0 / unlimited).  Returns ranks (host).
  void run(const NodesView& S, const NodesView& E1, bool e1s, const NodesView& E2, bool e2s,
           double tol_rel, const std::vector<double>& tol_abs, const std::vector<int>& subset,
           const std::vector<int>& min_rank, const std::vector<int>& max_rank, unsigned long long seed,
           cudaStream_t s);
  // P_j (m_j x rank_j, ld ldp_j) for every job with a non-null target.
  void interp(const std::vector<double*>& P, const std::vector<int>& ldp, cudaStream_t s);
  std::vector<int> pivots(cudaStream_t s) const;  // concatenated, offsets moff
  size_t piv_off(int j) const { return jobs[j].moff; }
};

// Hierarchical row ID of a tall matrix Y (rows = `rows`, DOFs of node set S;
// columns given by a column spec as in IdMatProb): chunks of `chunk` rows are
// decomposed independently and merged pairwise up a binary tree, so that the
// cost stays linear in the number of rows (Sec. 3.3, the hierarchical ID of the
// far field); once a level has few problems, one root over all of their
// skeletons (a single wide problem for the grid-wide factorisation) ends the
// tree.  Absolute tolerance = tol * max row norm of Y (Def. 3.1 with
// ||Y|| bounded below by its largest row norm).
struct TreeId {
  int k = 0;
  std::vector<int> skel;  // positions into `rows` of the skeleton rows
  DBuf<double> P;         // m x k interpolation matrix, P[skel] = I (not formed when deferred)
  // The tree's levels and their interpolation matrices: expand() forms
  // P T (m x kout) for a k x kout matrix T (leading dimension ldT; null T:
  // the identity, kout = k) by the top-down products, so that a later
  // right factor (a recompression) costs products with kout columns only.
  struct Levels;
  std::shared_ptr<Levels> lv;
  DBuf<double> expand(const double* T, int ldT, int kout, cudaStream_t s) const;
};
// defer: return the levels without forming P (see TreeId::expand).
TreeId tree_row_id(const NodesView& S, const std::vector<int>& rows, const IdMatProb& colspec,
                   const NodesView& E1, bool e1s, const NodesView& E2, bool e2s, double tol,
                   int sketch_cols, int sketch_width, unsigned long long seed, int chunk,
                   cudaStream_t s, bool defer = false);

struct HbsNode {
  int lo = 0, hi = 0;  // point range
  int k = 0;           // rank (skeleton size)
  int m = 0;           // candidate count (rows of U, V, E, F^T, G)
  std::vector<int> skr, skc;  // skeleton DOFs (rows / columns)
};

class Hbs {
 public:
  int N = 0, L = 0;
  std::vector<HbsNode> node;  // heap order, index 1 .. 2^{L+1}-1
  // per-level storage (index = level)
  struct Level {
    DBuf<double> U, Vt, E, F, G, B, D;  // F holds F* (k x m)
    std::vector<size_t> oU, oVt, oE, oF, oG, oB12, oB21, oD;
    std::vector<int> koff;  // prefix sums of ranks at this level (size nn+1)
    DBuf<float> G32, E32, F32;
    DBuf<__nv_bfloat16> G16, E16, F16;  // BF16 copies (preconditioner sweeps)
    mutable DBuf<float2> U2, Vt2, B2, D2;  // double-FP32 copies of the forward factors (made on first use)
    mutable DBuf<float> Uf, Vtf, Bf, Df;   // FP32 copies of the forward factors (made on first use)
    mutable DBuf<float2> E2, F2, G2;       // double-FP32 copies of the inverse factors (made on first use)
  };
  std::vector<Level> lev;
  long long inv_elems = 0, fwd_elems = 0;
  size_t bytes = 0;
  int max_rank = 0;

  // Build from a node set (positions on host in `nodes.hx/hy` for planning):
  // compression level by level on s, each level's inverse on a second stream
  // as soon as that level is compressed (synchronised before returning).
  // fwd_only: the forward representation (U, V*, B, D) alone, no inverse.
  void build(const Nodes& nodes, const Opts& o, cudaStream_t s, bool fwd_only = false);
  // Single-leaf representation of a dense matrix A (2 npts x 2 npts, column
  // major; the handle takes it over): the forward apply uses A, the inverse
  // sweeps its inverse.  Throws RW_ERR_SINGULAR if A cannot be inverted.
  void build_dense(DBuf<double>&& A, int npts, cudaStream_t s);
  // x = A^{-1} b, b and x: 2N x nrhs (ld 2N).  Template on the sweep type.
  void apply_inverse(const double* b, double* x, int nrhs, cudaStream_t s) const;
  // the same as a sequence of per-level launches with per-call temporaries
  // (safe to call concurrently on one handle)
  void apply_inverse_levels(const double* b, double* x, int nrhs, cudaStream_t s) const {
    sweep_inverse<double>(b, x, nrhs, s);
  }
  void apply_inverse_f32(const float* b, float* x, int nrhs, cudaStream_t s) const;
  // BF16 matrices, FP32 vectors and accumulation (make_bf16 first)
  void apply_inverse_bf16(const float* b, float* x, int nrhs, cudaStream_t s) const;
  // y = A x via the forward representation.
  void apply_forward(const double* x, double* y, int nrhs, cudaStream_t s) const;
  // The same with the products in double-FP32 (copies made on first use).
  void apply_forward_df(const double* x, double* y, int nrhs, cudaStream_t s) const;
  // Copies and programs made after the build are allocated in stream order on
  // own_stream (a refined arc: its refinement's stream, which outlives it),
  // or with plain cudaMalloc when it is null (a shared wall, which any stream
  // may use and outlive).
  cudaStream_t own_stream = nullptr;
  void make_df(cudaStream_t s) const;
  mutable bool has_df = false;
  void make_df_inv(cudaStream_t s) const;
  mutable bool has_df_inv = false;
  void make_fp32_fwd(cudaStream_t s) const;
  mutable bool has_fp32_fwd = false;
  void make_fp32(cudaStream_t s);
  void make_bf16(cudaStream_t s);
  bool has_fp32 = false, has_bf16 = false;
  // Add the inverse sweep x = A^{-1} b to a program, starting at phase p0
  // (input and output addressed as program vectors); returns the next phase.
  int emit_inverse_sweep(Program& P, int p0, int in_b, long long in_o, int in_ld, int out_b, long long out_o,
                         int out_ld) const;
  // The same for the forward apply y = A x (V* up the tree, B across
  // siblings, U down, leaf D blocks), phases p0 .. p0 + 2L.
  int emit_forward_sweep(Program& P, int p0, int in_b, long long in_o, int in_ld, int out_b, long long out_o,
                         int out_ld) const;
  // single-launch inverse sweep on a program built on first use (bases:
  // b, x, workspace); same result as apply_inverse
  void apply_inverse_program(const double* b, double* x, int nrhs, cudaStream_t s) const;
  mutable Program inv_prog;
  mutable bool inv_prog_built = false;
  mutable DBuf<double> prog_ws;
  // Many right-hand sides: the forward apply and the inverse sweep as GEMM
  // programs (one persistent launch per 64 right-hand sides), emitted into a
  // caller's program or cached here.  atype (MA_*) picks the factors: FP64 or
  // double-FP32 for the forward apply (FP64 vectors), FP64, FP32 or BF16 for
  // the inverse (the program's vector type must match).  Bases: the input
  // at (xb, xo, ldx), the output at (yb, yo, ldy), temporaries in the
  // program's workspace; returns the next free phase.
  template <class GP>
  int emit_forward_g(GP& P, int p0, int xb, long long xo, int ldx, int yb, long long yo, int ldy, int atype) const;
  template <class GP>
  int emit_inverse_g(GP& P, int p0, int xb, long long xo, int ldx, int yb, long long yo, int ldy, int atype) const;
  mutable GProgram<double> gfwd64, gfwddf, ginv64, ginvdf;
  mutable GProgram<float> ginv32, ginv16;
  // one launch per 64 right-hand sides on the cached programs (built on first use)
  void forward_gemm(const double* x, double* y, int nrhs, bool df, cudaStream_t s) const;
  void inverse_gemm(const double* b, double* x, int nrhs, cudaStream_t s) const;
  // x = A^{-1} b with the sweep's products in double-FP32 (FP64 vectors; the
  // copies of E, F*, G are made on first use), any nrhs
  void inverse_gemm_df(const double* b, double* x, int nrhs, cudaStream_t s) const;
  void inverse_gemm_f32(const float* b, float* x, int nrhs, bool bf16, cudaStream_t s) const;

 private:
  template <class T, class MT = T>
  void sweep_inverse(const T* b, T* x, int nrhs, cudaStream_t s) const;
  template <class MT>
  void forward_impl(const double* x, double* y, int nrhs, cudaStream_t s) const;
};

}  // namespace rw
