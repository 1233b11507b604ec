// A "GEMV program": phases of independent small matrix-vector products,
// copies and fills over a few base buffers, executed by one persistent
// cooperative kernel with a grid-wide barrier between phases.  The HBS
// inverse sweep (leaves up, root, down) and the Woodbury correction are
// built once per handle as such a program, so a solve is a single launch
// with no host-side descriptor upload or allocation.
//
// Addressing: every vector is base[b] + off + r * ld for right-hand side r,
// with ld fixed per buffer (2N for caller vectors; the per-RHS block size for
// the workspace, whose right-hand sides are stored block after block), so a
// program does not depend on nrhs.
#pragma once
#include "dense.cuh"

namespace rw {

enum { OP_GEMV = 0, OP_COPY = 1, OP_ZERO = 2, OP_REDUCE = 3 };
constexpr int kMaxBases = 4;

struct GOp {
  int kind;
  int m, n;          // GEMV: A is m x n; COPY/ZERO: m entries; REDUCE: m entries, n parts
  const double* A;   // GEMV matrix (absolute: matrices never move after a build)
  int lda;
  int xb, ldx;       // x = base[xb] + xo (+ r * ldx)
  long long xo;
  int yb, ldy;       // y = base[yb] + yo (+ r * ldy)
  long long yo;
  const int* ix;     // COPY: y[iy[i]] = x[ix[i]] (null = identity); ZERO: y[iy[i]] = 0
  const int* iy;
  double alpha, beta;
};

class Program {
 public:
  // add ops to phase p (phases are created on demand; phase p+1 runs after
  // every op of phase p has finished)
  void gemv(int p, const double* A, int m, int n, int lda, int xb, long long xo, int ldx, int yb, long long yo,
            int ldy, double alpha, double beta);
  void copy(int p, int n, int xb, long long xo, int ldx, const int* ix, int yb, long long yo, int ldy,
            const int* iy);
  void zero(int p, int n, int yb, long long yo, int ldy, const int* iy);
  long long ws_alloc(long long elems);  // workspace offset within one RHS block
  long long ws_per_rhs() const { return ws_; }
  int nphases() const { return int(phases_.size()); }
  void finalize(cudaStream_t s);        // split wide GEMVs, tile, upload
  // Execute on bases[0..kMaxBases) for nrhs right-hand sides.
  void run(double* const* bases, int nrhs, cudaStream_t s) const;
  long long matrix_elems() const { return mat_elems_; }
  int launches_per_run(int nrhs) const { return (nrhs + 7) / 8; }
  // Autotuner: times the three GEMV tile heights (16, 32, 64 rows) on these
  // bases and keeps the fastest; returns its time (ms).
  float autotune(double* const* bases, int nrhs, cudaStream_t s);
  int tile_rows() const { return tr_index_ == 0 ? 16 : tr_index_ == 2 ? 64 : 32; }
  void set_tile_rows(int tr) { tr_index_ = tr == 16 ? 0 : tr == 64 ? 2 : 1; }

 private:
  std::vector<std::vector<GOp>> phases_;
  long long ws_ = 0, mat_elems_ = 0;
  int nph_ = 0;
  int grid_[3] = {0, 0, 0};
  int tr_index_ = 1;
  DBuf<GOp> d_ops_;
  DBuf<int> d_tile_[3], d_top_[3], d_phase_;
  // L2 prefetch list: contiguous byte ranges of every phase's matrices
  // (16-byte aligned, at most kPrefetchChunk bytes each), phase p's ranges at
  // [d_pf_off_[p], d_pf_off_[p+1])
  DBuf<const char*> d_pf_addr_;
  DBuf<int> d_pf_bytes_, d_pf_off_;
};

}  // namespace rw
