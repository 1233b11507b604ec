// A "GEMM program": the matrix-matrix counterpart of the GEMV program
// (program.cuh) for many right-hand sides.  Phases of independent small
// products C = alpha A X + beta C (A a stored factor, X and C blocks of
// vectors, one column per right-hand side), copies, fills and split-K
// reductions over a few base buffers, executed by one persistent cooperative
// kernel with a grid-wide barrier between phases.  Each product is cut into
// output tiles of 64 rows x 64 right-hand sides; a launch covers up to 64
// right-hand sides (more take one launch per 64).  A program over FP64
// vectors takes FP64 factors or their double-FP32 copies (float2, products
// and sums compensated to FP64-level accuracy); a program over FP32 vectors
// takes FP32 or BF16 factors with FP32 accumulation.  The HBS forward apply
// and inverse sweeps of a wall, of the refined arc and the Woodbury terms of
// a refinement become one launch per 64 right-hand sides this way, with no
// descriptor upload or allocation per solve.
//
// Addressing as in the GEMV program: vector i of a buffer is
// base[b] + off + r * ld for right-hand side r; the workspace base stores one
// block of ws_per_rhs() entries per right-hand side (ld = -1 when adding ops).
#pragma once
#include "dense.cuh"

namespace rw {

enum { MA_F64 = 0, MA_F32 = 1, MA_BF16 = 2, MA_DF = 3 };
enum { MOP_GEMM = 0, MOP_COPY = 1, MOP_ZERO = 2, MOP_REDUCE = 3 };
constexpr int kGBases = 6;

struct MOp {
  int kind;
  int m, n;         // GEMM: A is m x n; COPY/ZERO: m entries; REDUCE: m entries, n parts
  const void* A;    // GEMM matrix (absolute: factors never move after a build)
  int lda, atype;   // atype: MA_*
  int xb, ldx;      // x = base[xb] + xo (+ r * ldx)
  long long xo;
  int yb, ldy;      // y = base[yb] + yo (+ r * ldy)
  long long yo;
  const int* ix;    // COPY: y[iy[i]] = x[ix[i]] (null = identity); ZERO: y[iy[i]] = 0
  const int* iy;
  double alpha, beta;
};

template <class T>  // vector type: double or float
class GProgram {
 public:
  explicit GProgram(int ws_base = 2) : wsb_(ws_base) {}
  void gemm(int p, const double* A, int m, int n, int lda, int xb, long long xo, int ldx, int yb, long long yo,
            int ldy, double alpha, double beta) { add_gemm(p, A, MA_F64, m, n, lda, xb, xo, ldx, yb, yo, ldy, alpha, beta); }
  void gemm(int p, const float2* A, int m, int n, int lda, int xb, long long xo, int ldx, int yb, long long yo,
            int ldy, double alpha, double beta) { add_gemm(p, A, MA_DF, m, n, lda, xb, xo, ldx, yb, yo, ldy, alpha, beta); }
  void gemm(int p, const float* A, int m, int n, int lda, int xb, long long xo, int ldx, int yb, long long yo,
            int ldy, double alpha, double beta) { add_gemm(p, A, MA_F32, m, n, lda, xb, xo, ldx, yb, yo, ldy, alpha, beta); }
  void gemm(int p, const __nv_bfloat16* A, int m, int n, int lda, int xb, long long xo, int ldx, int yb,
            long long yo, int ldy, double alpha, double beta) {
    add_gemm(p, A, MA_BF16, m, n, lda, xb, xo, ldx, yb, yo, ldy, alpha, beta);
  }
  void copy(int p, int n, int xb, long long xo, int ldx, const int* ix, int yb, long long yo, int ldy,
            const int* iy);
  void zero(int p, int n, int yb, long long yo, int ldy, const int* iy);
  long long ws_alloc(long long elems);  // workspace offset within one RHS block
  long long ws_per_rhs() const { return ws_; }
  int ws_base() const { return wsb_; }
  int nphases() const { return int(phases_.size()); }
  bool finalized() const { return done_; }
  // split long inner dimensions, tile, upload.  The program's device tables
  // are allocated in stream order on `alloc` (the owner's stream, which must
  // outlive the program), or with plain cudaMalloc when it is null (programs
  // of a shared wall, which any stream may use and outlive).
  void finalize(cudaStream_t s, cudaStream_t alloc = nullptr);
  // Execute on bases[0..kGBases) for nrhs right-hand sides (the workspace
  // base must hold ws_per_rhs() * nrhs entries).
  void run(T* const* bases, int nrhs, cudaStream_t s) const;
  double flops_per_rhs() const { return flops_; }  // 2 * sum of m * n over the products

 private:
  void add_gemm(int p, const void* A, int atype, int m, int n, int lda, int xb, long long xo, int ldx, int yb,
                long long yo, int ldy, double alpha, double beta);
  std::vector<std::vector<MOp>> phases_;
  long long ws_ = 0;
  int wsb_ = 2;
  int nph_ = 0, grid_ = 0;
  bool done_ = false;
  bool prof_class_df_ = false;
  int tk_ = -1;  // tile kind of the program's products (one per program)
  std::vector<int> ph_tiles_;
  std::vector<double> ph_mac_;   // multiply-adds per right-hand side of each phase (diagnostics)
  std::vector<int> ph_kmax_;     // longest inner dimension of a tile in each phase (diagnostics)
  double flops_ = 0.0;
  DBuf<MOp> d_ops_;
  DBuf<int> d_tile0_, d_top_, d_phase_;
};

}  // namespace rw
