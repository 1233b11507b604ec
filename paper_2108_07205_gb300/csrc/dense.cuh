// Batched dense FP64 (and FP32) building blocks of the rwsolve library.
// Every routine takes a list of independent problems of varying size and
// runs them in one launch; matrices are column-major.
#pragma once
#include <cuda_bf16.h>
#include "rw_common.cuh"

namespace rw {

// C (m x n) = alpha op(A) op(B) + beta C, op(A): m x k, op(B): k x n.
struct GemmProb {
  const double* A;
  const double* B;
  double* C;
  int m, n, k;
  int lda, ldb, ldc;
  int ta, tb;  // 0 = as stored, 1 = transposed
  double alpha, beta;
};
void batched_gemm(const std::vector<GemmProb>& probs, cudaStream_t s);

// y (m x nrhs) = alpha A x + beta y for column-major A (m x n) and a few
// right-hand sides (nrhs <= 8).  Vector type T (double or float) and matrix
// type MT (T, or __nv_bfloat16 with float vectors); accumulation is in T.
// When a problem is wide (n large and m small) the columns are split into
// chunks whose partial sums go to a scratch buffer and are added in a fixed
// order (deterministic).
template <class T, class MT = T>
struct GemvProb {
  const MT* A;
  const T* x;
  T* y;
  int m, n, lda, ldx, ldy;
  double alpha, beta;
};

// Scratch needed by batched_gemv for a problem list (in elements of T).
template <class T, class MT = T>
size_t gemv_scratch_elems(const std::vector<GemvProb<T, MT>>& probs, int nrhs);

// Runs the problems; `scratch` must hold gemv_scratch_elems() elements (may
// be null when that is 0).
template <class T, class MT = T>
void batched_gemv(const std::vector<GemvProb<T, MT>>& probs, int nrhs, T* scratch,
                  cudaStream_t s);

// The same GEMV launch with caller-provided device memory for the launch
// descriptors (desc, gemv_into_sizes bytes, 16-byte aligned) and the split-K
// partials (scratch, gemv_into_sizes elements): performs no allocation.
template <class T>
void gemv_into_sizes(const std::vector<GemvProb<T>>& probs, int nrhs, size_t* desc_bytes, size_t* scratch_elems);
template <class T>
void gemv_into(const std::vector<GemvProb<T>>& probs, int nrhs, void* desc, T* scratch, cudaStream_t s);

// y = alpha A x + beta y for a problem list and any nrhs: GEMV kernels for
// nrhs <= 8, the tiled GEMMs above that (FP64, FP32 accumulation for FP32 and
// BF16 matrices, double-FP32 for float2 matrices with FP64 vectors).
// Temporaries are stream-ordered.
template <class T, class MT = T>
void matvec(const std::vector<GemvProb<T, MT>>& probs, int nrhs, cudaStream_t s);

// Batched GEMM with FP32 accumulation for the low-precision sweeps with many
// right-hand sides: C (m x n, float) = alpha A B + beta C with A column-major
// in MT (float, or __nv_bfloat16 widened as it is read) and B float.  Same
// tiling and split-K rule as batched_gemm; split partial sums are added in a
// fixed order.
template <class MT>
struct GemmF32Prob {
  const MT* A;
  const float* B;
  float* C;
  int m, n, k;
  int lda, ldb, ldc;
  float alpha, beta;
};
template <class MT>
void batched_gemm_f32(const std::vector<GemmF32Prob<MT>>& probs, cudaStream_t s);

// Double-FP32 ("df") matrices: an FP64 matrix held as the FP32 pairs
// (hi, lo) = (fl32(a), fl32(a - hi)), interleaved as float2.  hi + lo carries
// 48 bits of a's significand (relative error <= 2^-48 ~ 3.6e-15).
void copy_d2df(const double* in, float2* out, size_t n, cudaStream_t s);
// C (m x n, FP64) = alpha A B + beta C with A df (column-major) and B FP64
// (split into df pairs as it is read).  Every product is formed exactly from
// FP32 operations (the rounding error of hi * hi by an FMA, the cross terms
// hi * lo by FMAs), sums are compensated (two-sum of the hi products, the
// errors and cross terms in a second FP32 accumulator) and flushed to FP64
// every 128 terms of the inner dimension, so the result keeps FP64-level
// accuracy (~1e-14 relative per product) while running on the FP32 units.
struct GemmDfProb {
  const float2* A;
  const double* B;
  double* C;
  int m, n, k;
  int lda, ldb, ldc;
  double alpha, beta;
};
void batched_gemm_df(const std::vector<GemmDfProb>& probs, cudaStream_t s);

// Inverse of square matrices by Gauss-Jordan elimination with partial
// pivoting (the pivot sequence of LU with partial pivoting).  A is read, Ainv
// written (may not alias), W is an n*n work copy.  flag[i] set to 1 if a
// pivot fell below 1e-14 * max|A|.
struct InvProb {
  const double* A;
  double* Ainv;
  double* W;
  int n, lda, ldinv;
  int* flag;
};
void batched_inverse(const std::vector<InvProb>& probs, cudaStream_t s);

// Inverse of one large square matrix (n x n, column major, ld n) by block
// Gauss-Jordan elimination: for each diagonal block of at most nb rows, its
// inverse (Gauss-Jordan with partial pivoting inside the block) scales the
// block row and GEMMs eliminate the block column from every other row.  No
// pivoting across blocks: meant for matrices whose diagonal blocks and their
// Schur complements stay well conditioned (second-kind operators such as the
// dense hole matrix).  A is not modified; flag is set if a pivot is tiny.
void block_inverse(const double* A, double* Ainv, int n, int nb, int* flag, cudaStream_t s);

// Interpolative decomposition on the columns of W (the rows of Y = W^T) by
// column-pivoted Householder QR (Def. 3.1): W (nr x nc) is overwritten;
// stop when the largest remaining column norm is <= max(tol_abs,
// tol_rel * first pivot norm) once at least min_rank steps were taken, or at
// max_rank.  A min_rank above the numerical rank is met by taking further
// candidates in pivot order as skeletons with zero coefficients.  The last
// four norms entries hold the number of usable pivots and the layout.  Outputs rank k, the pivot order piv (nc), and the interpolation
// matrix P (nc x k, column-major, leading dimension ldp) with
// Y ~= P Y(piv[0:k], :) and P(piv[i], :) = e_i.
struct IdProb {
  double* W;
  int ldw, nr, nc;
  double tol_abs, tol_rel;
  int min_rank, max_rank;
  int* piv;
  double* norms;  // id_norms_elems(nc) work entries
  double* P;
  int ldp;
  int* rank;
};
// Work entries needed in IdProb::norms for a problem with nc candidates.
inline size_t id_norms_elems(int nc) { return 2 * size_t(nc) + 4; }
// paired: probs[2i] and probs[2i+1] are factorised together with a joint
// stopping rule (both end at the larger of their two ranks).
void batched_id(const std::vector<IdProb>& probs, cudaStream_t s, bool paired = false);
// True when one problem of nr x nc goes to the grid-wide factorisation
// (batched_id with a single problem).
bool grid_id_fits(int nr, int nc);

// Writes P (nc x rank) for factorisations finished by batched_id (P may have
// been null there).  max_elems bounds nc * rank over the list.
void batched_id_interp(const std::vector<IdProb>& probs, int max_elems, cudaStream_t s);

// Fill a buffer with random +-1 entries from a counter-based hash of
// (seed, index) (splitmix64 finaliser).
void fill_rademacher(double* out, size_t n, unsigned long long seed, cudaStream_t s);

// Elementwise helpers.
void fill_zero(double* p, size_t n, cudaStream_t s);
void axpby(const double* x, double* y, size_t n, double a, double b, cudaStream_t s);  // y = a x + b y
void copy_d2f(const double* in, float* out, size_t n, cudaStream_t s);
// out = bf16(in), round to nearest even
void copy_d2bf(const double* in, __nv_bfloat16* out, size_t n, cudaStream_t s);

}  // namespace rw
