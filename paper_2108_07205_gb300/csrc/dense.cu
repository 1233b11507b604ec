// Batched dense kernels: tiled GEMM, small-RHS GEMV with deterministic
// split-K, Gauss-Jordan inverse, column-pivoted QR interpolative
// decomposition, and fills.  One launch per problem list; each CTA finds its
// problem from a prefix sum of per-problem tile counts.
#include "dense.cuh"
#include <algorithm>
#include <cmath>

namespace rw {

namespace {

__device__ __forceinline__ int find_problem(const int* offs, int nprob, int tile) {
  // offs: nprob + 1 prefix sums; returns b with offs[b] <= tile < offs[b+1]
  int lo = 0, hi = nprob;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (offs[mid] <= tile) lo = mid; else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------------ GEMM
constexpr int GBM = 64, GBN = 64, GBK = 16;

__global__ void __launch_bounds__(256) k_gemm(const GemmProb* probs, const int* offs, int nprob) {
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  const int tile = blockIdx.x;
  const int b = find_problem(offs, nprob, tile);
  const GemmProb P = probs[b];
  const int tilesM = (P.m + GBM - 1) / GBM;
  const int t = tile - offs[b];
  const int m0 = (t % tilesM) * GBM, n0 = (t / tilesM) * GBN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < P.k; k0 += GBK) {
    // load op(A)[m0 : m0+64, k0 : k0+16]
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * 256;  // 0..1023
      int i, kk;
      if (!P.ta) { i = e & 63; kk = e >> 6; } else { kk = e & 15; i = e >> 4; }
      int gi = m0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < P.m && gk < P.k)
        v = P.ta ? P.A[gk + size_t(gi) * P.lda] : P.A[gi + size_t(gk) * P.lda];
      As[kk][i] = v;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * 256;
      int j, kk;
      if (!P.tb) { kk = e & 15; j = e >> 4; } else { j = e & 63; kk = e >> 6; }
      int gj = n0 + j, gk = k0 + kk;
      double v = 0.0;
      if (gj < P.n && gk < P.k)
        v = P.tb ? P.B[gj + size_t(gk) * P.ldb] : P.B[gk + size_t(gj) * P.ldb];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gi = m0 + ty + 16 * i;
    if (gi >= P.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gj = n0 + tx + 16 * j;
      if (gj >= P.n) continue;
      double* c = P.C + gi + size_t(gj) * P.ldc;
      double v = P.alpha * acc[i][j];
      if (P.beta != 0.0) v += P.beta * *c;
      *c = v;
    }
  }
}

// ------------------------------------------------------------------ GEMV
// Tile = 64 rows x one column chunk; 256 threads = 64 rows x 4 column lanes.
constexpr int VR = 64;
constexpr int VCHUNK = 2048;  // columns per split-K chunk

template <class T>
struct GemvWork {  // device-side descriptor (adds split-K bookkeeping)
  GemvProb<T> p;
  int tilesM, nchunk;
  long long scratch_off;  // offset of this problem's partials (elements)
};

template <class T> struct Acc { typedef double type; };
template <> struct Acc<float> { typedef float type; };

template <class T, int NR>
__global__ void __launch_bounds__(256) k_gemv(const GemvWork<T>* work, const int* offs, int nprob,
                                              T* scratch) {
  typedef typename Acc<T>::type A_t;
  const int tile = blockIdx.x;
  const int b = find_problem(offs, nprob, tile);
  const GemvWork<T> W = work[b];
  const GemvProb<T>& P = W.p;
  const int t = tile - offs[b];
  const int mt = t % W.tilesM, chunk = t / W.tilesM;
  const int r0 = mt * VR;
  const int c0 = chunk * VCHUNK, c1 = min(P.n, c0 + VCHUNK);
  const int lr = threadIdx.x & 63, lc = threadIdx.x >> 6;  // row, column lane
  const int row = r0 + lr;
  A_t acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = A_t(0);
  __shared__ A_t xs[256][NR];
  for (int cb = c0; cb < c1; cb += 256) {
    const int ncur = min(256, c1 - cb);
    __syncthreads();
    for (int e = threadIdx.x; e < ncur; e += 256)
#pragma unroll
      for (int r = 0; r < NR; ++r) xs[e][r] = A_t(P.x[cb + e + size_t(r) * P.ldx]);
    __syncthreads();
    if (row < P.m) {
      const T* a = P.A + row + size_t(cb) * P.lda;
      for (int j = lc; j < ncur; j += 4) {
        const A_t v = A_t(a[size_t(j) * P.lda]);
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = fma(v, xs[j][r], acc[r]);
      }
    }
  }
  __shared__ A_t red[4][64][NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) red[lc][lr][r] = acc[r];
  __syncthreads();
  if (lc == 0 && row < P.m) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      A_t s = red[0][lr][r] + red[1][lr][r] + red[2][lr][r] + red[3][lr][r];
      if (W.nchunk == 1) {
        T* y = P.y + row + size_t(r) * P.ldy;
        A_t v = A_t(P.alpha) * s;
        if (P.beta != 0.0) v += A_t(P.beta) * A_t(*y);
        *y = T(v);
      } else {
        scratch[W.scratch_off + (size_t(chunk) * NR + r) * P.m + row] = T(s);
      }
    }
  }
}

template <class T, int NR>
__global__ void k_gemv_reduce(const GemvWork<T>* work, int nprob, const T* scratch) {
  typedef typename Acc<T>::type A_t;
  const int b = blockIdx.y;
  const GemvWork<T> W = work[b];
  if (W.nchunk == 1) return;
  const GemvProb<T>& P = W.p;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < P.m; row += gridDim.x * blockDim.x) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      A_t s = 0;
      for (int c = 0; c < W.nchunk; ++c) s += A_t(scratch[W.scratch_off + (size_t(c) * NR + r) * P.m + row]);
      T* y = P.y + row + size_t(r) * P.ldy;
      A_t v = A_t(P.alpha) * s;
      if (P.beta != 0.0) v += A_t(P.beta) * A_t(*y);
      *y = T(v);
    }
  }
}

// ------------------------------------------------------------------ inverse
__device__ double block_reduce_max_abs_arg(double v, int idx, int* arg_out, double* sval, int* sidx) {
  // returns max |v| over the block and its index (smallest index on ties)
  const int tid = threadIdx.x;
  for (int off = 16; off > 0; off >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, v, off);
    int oi = __shfl_down_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if ((tid & 31) == 0) { sval[tid >> 5] = v; sidx[tid >> 5] = idx; }
  __syncthreads();
  if (tid < 32) {
    int nw = blockDim.x >> 5;
    v = tid < nw ? sval[tid] : -1.0;
    idx = tid < nw ? sidx[tid] : 0x7fffffff;
    for (int off = 16; off > 0; off >>= 1) {
      double ov = __shfl_down_sync(0xffffffffu, v, off);
      int oi = __shfl_down_sync(0xffffffffu, idx, off);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (tid == 0) { sval[0] = v; sidx[0] = idx; }
  }
  __syncthreads();
  double r = sval[0];
  *arg_out = sidx[0];
  __syncthreads();
  return r;
}

__device__ double block_reduce_sum(double v, double* sbuf) {
  const int tid = threadIdx.x;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((tid & 31) == 0) sbuf[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    int nw = blockDim.x >> 5;
    v = tid < nw ? sbuf[tid] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (tid == 0) sbuf[0] = v;
  }
  __syncthreads();
  double r = sbuf[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(512) k_inverse(const InvProb* probs) {
  const InvProb P = probs[blockIdx.x];
  const int n = P.n, tid = threadIdx.x, nt = blockDim.x;
  double* W = P.W;  // ld = n
  double* X = P.Ainv;
  __shared__ double sval[32];
  __shared__ int sidx[32];
  __shared__ int s_flag;
  extern __shared__ double colc[];  // pivot column multipliers (n)
  if (tid == 0) s_flag = 0;
  double amax = 0.0;
  for (int e = tid; e < n * n; e += nt) {
    int i = e % n, j = e / n;
    double v = P.A[i + size_t(j) * P.lda];
    W[e] = v;
    X[i + size_t(j) * P.ldinv] = (i == j) ? 1.0 : 0.0;
    amax = fmax(amax, fabs(v));
  }
  int dummy;
  amax = block_reduce_max_abs_arg(amax, 0, &dummy, sval, sidx);
  const double tiny = 1e-14 * amax;
  for (int c = 0; c < n; ++c) {
    double v = -1.0;
    int idx = 0x7fffffff;
    for (int r = c + tid; r < n; r += nt) {
      double a = fabs(W[r + size_t(c) * n]);
      if (a > v) { v = a; idx = r; }
    }
    int p;
    double pv = block_reduce_max_abs_arg(v, idx, &p, sval, sidx);
    if (!(pv > tiny)) { if (tid == 0) s_flag = 1; if (pv == 0.0) { __syncthreads(); break; } }
    if (p != c) {
      for (int j = tid; j < n; j += nt) {
        double t1 = W[c + size_t(j) * n]; W[c + size_t(j) * n] = W[p + size_t(j) * n]; W[p + size_t(j) * n] = t1;
        double t2 = X[c + size_t(j) * P.ldinv]; X[c + size_t(j) * P.ldinv] = X[p + size_t(j) * P.ldinv]; X[p + size_t(j) * P.ldinv] = t2;
      }
      __syncthreads();
    }
    const double inv = 1.0 / W[c + size_t(c) * n];
    __syncthreads();
    // scale pivot row; save multipliers
    for (int j = tid; j < n; j += nt) {
      W[c + size_t(j) * n] *= inv;
      X[c + size_t(j) * P.ldinv] *= inv;
    }
    for (int r = tid; r < n; r += nt) colc[r] = (r == c) ? 0.0 : W[r + size_t(c) * n];
    __syncthreads();
    // eliminate column c from every other row (rows fastest: coalesced)
    const int ncw = n - c - 1;
    for (int e = tid; e < n * ncw; e += nt) {
      const int r = e % n, j = c + 1 + e / n;
      if (r != c) W[r + size_t(j) * n] -= colc[r] * W[c + size_t(j) * n];
    }
    for (int e = tid; e < n * n; e += nt) {
      const int r = e % n, j = e / n;
      if (r != c) X[r + size_t(j) * P.ldinv] -= colc[r] * X[c + size_t(j) * P.ldinv];
    }
    __syncthreads();
  }
  if (tid == 0 && P.flag) *P.flag = s_flag;
}

// ------------------------------------------------------------------ ID
__global__ void __launch_bounds__(256) k_cpqr_id(const IdProb* probs) {
  const IdProb P = probs[blockIdx.x];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int nr = P.nr, nc = P.nc, ld = P.ldw;
  double* W = P.W;
  double* nrm = P.norms;
  double* nrm0 = P.norms + nc;
  int* piv = P.piv;
  __shared__ double sval[32];
  __shared__ int sidx[32];
  __shared__ double s_tau;
  if (nr <= 0 || nc <= 0) { if (tid == 0) *P.rank = 0; return; }
  for (int j = tid; j < nc; j += nt) piv[j] = j;
  for (int j = warp; j < nc; j += nw) {
    double s = 0.0;
    for (int i = lane; i < nr; i += 32) { double v = W[i + size_t(j) * ld]; s += v * v; }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) { nrm[j] = sqrt(s); nrm0[j] = nrm[j]; }
  }
  __syncthreads();
  const int maxsteps = min(min(nr, nc), P.max_rank);
  double ref = 0.0;
  int s = 0;
  const double tol3z = sqrt(2.220446049250313e-16);
  for (; s < maxsteps; ++s) {
    double v = -1.0;
    int idx = 0x7fffffff;
    for (int j = s + tid; j < nc; j += nt) if (nrm[j] > v) { v = nrm[j]; idx = j; }
    int p;
    double vmax = block_reduce_max_abs_arg(v, idx, &p, sval, sidx);
    if (s == 0) ref = vmax;
    const double thr = fmax(P.tol_abs, P.tol_rel * ref);
    if (vmax <= 0.0 || (s >= P.min_rank && vmax <= thr)) break;
    if (p != s) {
      for (int i = tid; i < nr; i += nt) {
        double t1 = W[i + size_t(s) * ld]; W[i + size_t(s) * ld] = W[i + size_t(p) * ld]; W[i + size_t(p) * ld] = t1;
      }
      if (tid == 0) {
        double t = nrm[s]; nrm[s] = nrm[p]; nrm[p] = t;
        t = nrm0[s]; nrm0[s] = nrm0[p]; nrm0[p] = t;
        int q = piv[s]; piv[s] = piv[p]; piv[p] = q;
      }
      __syncthreads();
    }
    // Householder vector for W[s:nr, s]
    double* col = W + size_t(s) * ld;
    double part = 0.0;
    for (int i = s + 1 + tid; i < nr; i += nt) part += col[i] * col[i];
    const double xn2 = block_reduce_sum(part, sval);
    const double alpha = col[s];
    if (tid == 0) {
      if (xn2 == 0.0) {
        s_tau = 0.0;  // already triangular in this column
      } else {
        double beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
        s_tau = (beta - alpha) / beta;
        sval[1] = 1.0 / (alpha - beta);
        col[s] = beta;
      }
    }
    __syncthreads();
    const double tau = s_tau;
    if (tau != 0.0) {
      const double sc = sval[1];
      for (int i = s + 1 + tid; i < nr; i += nt) col[i] *= sc;
    }
    __syncthreads();
    // apply H = I - tau v v^T (v_s = 1) to columns s+1..nc-1, update norms
    for (int j = s + 1 + warp; j < nc; j += nw) {
      double* cj = W + size_t(j) * ld;
      if (tau != 0.0) {
        double d = 0.0;
        for (int i = s + 1 + lane; i < nr; i += 32) d += col[i] * cj[i];
        for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
        d = __shfl_sync(0xffffffffu, d, 0);
        d = tau * (d + cj[s]);
        for (int i = s + 1 + lane; i < nr; i += 32) cj[i] -= d * col[i];
        __syncwarp();
        if (lane == 0) cj[s] -= d;
        __syncwarp();
      }
      // norm downdate (LAPACK xLAQP2 scheme)
      double nj = nrm[j];
      int recompute = 0;
      if (nj != 0.0) {
        double t = fabs(cj[s]) / nj;
        t = fmax(0.0, (1.0 + t) * (1.0 - t));
        double r = nj / nrm0[j];
        double t2 = t * r * r;
        if (t2 <= tol3z) recompute = 1;
        else if (lane == 0) nrm[j] = nj * sqrt(t);
      }
      if (recompute) {
        double q = 0.0;
        for (int i = s + 1 + lane; i < nr; i += 32) q += cj[i] * cj[i];
        for (int off = 16; off > 0; off >>= 1) q += __shfl_down_sync(0xffffffffu, q, off);
        if (lane == 0) { nrm[j] = sqrt(q); nrm0[j] = nrm[j]; }
      }
      __syncwarp();
    }
    __syncthreads();
  }
  // Fixed-rank requests beyond the numerical rank take further candidates in
  // pivot order as skeletons with zero interpolation coefficients.
  const int k = max(s, min(P.min_rank, nc));
  int keff = s;
  for (int i = 0; i < s; ++i)
    if (!(fabs(W[i + size_t(i) * ld]) > 1e-15 * ref)) { keff = i; break; }
  // T = R11^{-1} R12 over the first keff pivots, in place in W[0:keff, k:nc];
  // rows keff..k-1 of T are zero.
  for (int j = k + tid; j < nc; j += nt) {
    double* cj = W + size_t(j) * ld;
    for (int i = keff - 1; i >= 0; --i) {
      double acc = cj[i];
      for (int l = i + 1; l < keff; ++l) acc -= W[i + size_t(l) * ld] * cj[l];
      cj[i] = acc / W[i + size_t(i) * ld];
    }
    for (int i = keff; i < k && i < nr; ++i) cj[i] = 0.0;
  }
  if (tid == 0) { *P.rank = k; P.norms[0] = double(keff); }
  __syncthreads();
  if (P.P) {
    for (int e = tid; e < nc * k; e += nt) {
      int j = e % nc, c = e / nc;
      double v;
      if (j < k) v = (j == c) ? 1.0 : 0.0;
      else v = (c < keff) ? W[c + size_t(j) * ld] : 0.0;
      P.P[piv[j] + size_t(c) * P.ldp] = v;
    }
  }
}

// Interpolation matrix from a finished factorisation (rank in *rank, number
// of usable pivots in norms[0]).
__global__ void k_id_interp(const IdProb* probs) {
  const IdProb P = probs[blockIdx.y];
  const int k = *P.rank, keff = int(P.norms[0]), nc = P.nc;
  const long long tot = (long long)nc * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int j = int(e % nc), c = int(e / nc);
    double v;
    if (j < k) v = (j == c) ? 1.0 : 0.0;
    else v = (c < keff) ? P.W[c + size_t(j) * P.ldw] : 0.0;
    P.P[P.piv[j] + size_t(c) * P.ldp] = v;
  }
}

__global__ void k_rademacher(double* out, size_t n, unsigned long long seed) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    out[i] = (z >> 63) ? 1.0 : -1.0;
  }
}

__global__ void k_fill_zero(double* p, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) p[i] = 0.0;
}
__global__ void k_d2f(const double* in, float* out, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) out[i] = float(in[i]);
}

int grid_for(size_t n) { return int(std::min<size_t>((n + 255) / 256, 152 * 16)); }

}  // namespace

void batched_gemm(const std::vector<GemmProb>& probs, cudaStream_t s) {
  std::vector<GemmProb> ps;
  std::vector<int> offs(1, 0);
  for (const auto& p : probs) {
    if (p.m <= 0 || p.n <= 0) continue;
    ps.push_back(p);
    int tiles = ceil_div(p.m, GBM) * ceil_div(p.n, GBN);
    offs.push_back(offs.back() + tiles);
  }
  if (ps.empty()) return;
  // k == 0 problems still need C = beta C: handled by the kernel (loop skipped)
  auto dp = to_device_tmp(ps, s);
  auto doff = to_device_tmp(offs, s);
  k_gemm<<<offs.back(), 256, 0, s>>>(dp.p, doff.p, int(ps.size()));
  RW_CHECK_LAUNCH();
}

template <class T>
static void gemv_plan(const std::vector<GemvProb<T>>& probs, int nrhs, std::vector<GemvWork<T>>& work,
                      std::vector<int>& offs, size_t& scratch) {
  offs.assign(1, 0);
  scratch = 0;
  for (const auto& p : probs) {
    if (p.m <= 0) continue;
    GemvWork<T> w;
    w.p = p;
    w.tilesM = ceil_div(p.m, VR);
    w.nchunk = std::max(1, ceil_div(std::max(p.n, 1), VCHUNK));
    w.scratch_off = (long long)scratch;
    if (w.nchunk > 1) scratch += size_t(w.nchunk) * nrhs * p.m;
    work.push_back(w);
    offs.push_back(offs.back() + w.tilesM * w.nchunk);
  }
}

template <class T>
size_t gemv_scratch_elems(const std::vector<GemvProb<T>>& probs, int nrhs) {
  std::vector<GemvWork<T>> w;
  std::vector<int> o;
  size_t sc;
  gemv_plan(probs, nrhs, w, o, sc);
  return sc;
}

template <class T>
void batched_gemv(const std::vector<GemvProb<T>>& probs, int nrhs, T* scratch, cudaStream_t s) {
  require(nrhs >= 1 && nrhs <= 8, "batched_gemv: nrhs must be in 1..8");
  std::vector<GemvWork<T>> work;
  std::vector<int> offs;
  size_t sc;
  gemv_plan(probs, nrhs, work, offs, sc);
  if (work.empty()) return;
  require(sc == 0 || scratch != nullptr, "batched_gemv: scratch buffer missing");
  auto dw = to_device_tmp(work, s);
  auto doff = to_device_tmp(offs, s);
  const int nprob = int(work.size());
  int maxm = 0;
  for (auto& w : work) maxm = std::max(maxm, w.p.m);
  switch (nrhs) {
#define RW_GEMV_CASE(NR)                                                                   \
  case NR:                                                                                 \
    k_gemv<T, NR><<<offs.back(), 256, 0, s>>>(dw.p, doff.p, nprob, scratch);               \
    if (sc) k_gemv_reduce<T, NR><<<dim3(ceil_div(maxm, 256), nprob), 256, 0, s>>>(dw.p, nprob, scratch); \
    break;
    RW_GEMV_CASE(1) RW_GEMV_CASE(2) RW_GEMV_CASE(3) RW_GEMV_CASE(4)
    RW_GEMV_CASE(5) RW_GEMV_CASE(6) RW_GEMV_CASE(7) RW_GEMV_CASE(8)
#undef RW_GEMV_CASE
  }
  RW_CHECK_LAUNCH();
}

template size_t gemv_scratch_elems<double>(const std::vector<GemvProb<double>>&, int);
template size_t gemv_scratch_elems<float>(const std::vector<GemvProb<float>>&, int);
template void batched_gemv<double>(const std::vector<GemvProb<double>>&, int, double*, cudaStream_t);
template void batched_gemv<float>(const std::vector<GemvProb<float>>&, int, float*, cudaStream_t);

template <>
void matvec<double>(const std::vector<GemvProb<double>>& probs, int nrhs, cudaStream_t s) {
  if (probs.empty() || nrhs <= 0) return;
  if (nrhs <= 8) {
    size_t sc = gemv_scratch_elems(probs, nrhs);
    TBuf<double> scratch(sc, s);
    batched_gemv(probs, nrhs, scratch.p, s);
  } else {
    std::vector<GemmProb> g;
    for (auto& p : probs) g.push_back(GemmProb{p.A, p.x, p.y, p.m, nrhs, p.n, p.lda, p.ldx, p.ldy, 0, 0, p.alpha, p.beta});
    batched_gemm(g, s);
  }
}

template <>
void matvec<float>(const std::vector<GemvProb<float>>& probs, int nrhs, cudaStream_t s) {
  if (probs.empty() || nrhs <= 0) return;
  for (int r0 = 0; r0 < nrhs; r0 += 8) {
    const int nr = std::min(8, nrhs - r0);
    std::vector<GemvProb<float>> ps = probs;
    for (auto& p : ps) { p.x += size_t(r0) * p.ldx; p.y += size_t(r0) * p.ldy; }
    size_t sc = gemv_scratch_elems(ps, nr);
    TBuf<float> scratch(sc, s);
    batched_gemv(ps, nr, scratch.p, s);
  }
}

void batched_inverse(const std::vector<InvProb>& probs, cudaStream_t s) {
  std::vector<InvProb> ps;
  int maxn = 0;
  for (auto& p : probs) if (p.n > 0) { ps.push_back(p); maxn = std::max(maxn, p.n); }
  if (ps.empty()) return;
  auto dp = to_device_tmp(ps, s);
  size_t smem = size_t(maxn) * sizeof(double);
  require(smem <= 200 * 1024, "batched_inverse: matrix too large");
  if (smem > 48 * 1024)
    RW_CUDA(cudaFuncSetAttribute(k_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  k_inverse<<<int(ps.size()), 512, smem, s>>>(dp.p);
  RW_CHECK_LAUNCH();
}

void batched_id(const std::vector<IdProb>& probs, cudaStream_t s) {
  if (probs.empty()) return;
  auto dp = to_device_tmp(probs, s);
  k_cpqr_id<<<int(probs.size()), 256, 0, s>>>(dp.p);
  RW_CHECK_LAUNCH();
}

void batched_id_interp(const std::vector<IdProb>& probs, int max_elems, cudaStream_t s) {
  if (probs.empty() || max_elems <= 0) return;
  auto dp = to_device_tmp(probs, s);
  k_id_interp<<<dim3(std::min(ceil_div(max_elems, 256), 1024), int(probs.size())), 256, 0, s>>>(dp.p);
  RW_CHECK_LAUNCH();
}

void fill_rademacher(double* out, size_t n, unsigned long long seed, cudaStream_t s) {
  if (!n) return;
  k_rademacher<<<grid_for(n), 256, 0, s>>>(out, n, seed);
  RW_CHECK_LAUNCH();
}
void fill_zero(double* p, size_t n, cudaStream_t s) {
  if (!n) return;
  k_fill_zero<<<grid_for(n), 256, 0, s>>>(p, n);
  RW_CHECK_LAUNCH();
}
void copy_d2f(const double* in, float* out, size_t n, cudaStream_t s) {
  if (!n) return;
  k_d2f<<<grid_for(n), 256, 0, s>>>(in, out, n);
  RW_CHECK_LAUNCH();
}

}  // namespace rw
