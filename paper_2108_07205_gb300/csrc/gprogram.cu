// Persistent cooperative executor of GEMM programs (see gprogram.cuh).
#include "gprogram.cuh"
#include "dfarith.cuh"
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <type_traits>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace rw {

namespace {

constexpr int GM = 64, GN = 64;   // output tile: 64 rows x 64 right-hand sides
constexpr int TE = 256;           // copy / fill / reduce: (entry, right-hand side) pairs per tile
// longest inner dimension one tile walks, by tile kind (a 64 x 64 x 16 FP64
// step is ~16 us of one SM's FP64 pipe, a double-FP32 64 x 32 x 16 step ~3 us)
constexpr int KMAX_F64 = 64, KMAX_DF = 128, KMAX_F32 = 256;
constexpr int kSmem = 16640;      // the largest tile layout below

template <class T>
struct GB { T* p[kGBases]; };

// ---- FP64 factors, FP64 vectors: K in steps of 16, the next step's tiles
// held in registers while the current one is multiplied
__device__ __forceinline__ void f64_load(const MOp& o, const double* A, const double* x, int m0, int k0, int K, int nc,
                                         double (&ra)[4], double (&rb)[4]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int e = tid + r * 256, i = e & 63, kk = e >> 6, gi = m0 + i, gk = k0 + kk;
    ra[r] = (gi < o.m && gk < K) ? A[gi + size_t(gk) * o.lda] : 0.0;
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int e = tid + r * 256, kk = e & 15, j = e >> 4, gk = k0 + kk;
    rb[r] = (j < nc && gk < K) ? x[gk + size_t(j) * o.ldx] : 0.0;
  }
}

__device__ void tile_f64(const MOp& o, int tile, const double* x, double* y, int nc, unsigned char* smem) {
  double (*As)[GM + 1] = reinterpret_cast<double (*)[GM + 1]>(smem);
  double (*Bs)[GN + 1] = reinterpret_cast<double (*)[GN + 1]>(smem + 16 * (GM + 1) * sizeof(double));
  const double* A = static_cast<const double*>(o.A);
  const int m0 = tile * GM, K = o.n;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  double ra[4], rb[4];
  f64_load(o, A, x, m0, 0, K, nc, ra, rb);
  for (int k0 = 0; k0 < K; k0 += 16) {
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * 256;
      As[e >> 6][e & 63] = ra[r];
      Bs[e & 15][e >> 4] = rb[r];
    }
    __syncthreads();
    if (k0 + 16 < K) f64_load(o, A, x, m0, k0 + 16, K, nc, ra, rb);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + ty + 16 * i;
    if (gi >= o.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = tx + 16 * j;
      if (gj >= nc) continue;
      double* yp = y + gi + size_t(gj) * o.ldy;
      double v = o.alpha * acc[i][j];
      if (o.beta != 0.0) v += o.beta * *yp;
      *yp = v;
    }
  }
  __syncthreads();
}

// ---- double-FP32 factors, FP64 vectors (split into pairs as they are
// staged): 64 rows x 32 right-hand sides per tile (two tiles across a launch's
// 64), 8 outputs per thread so that two CTAs fit an SM; K in steps of 16,
// compensated sums flushed every 128 terms
constexpr int DN = 32;

__device__ __forceinline__ void df_load(const MOp& o, const float2* A, const double* x, int m0, int n0, int k0, int K,
                                        int nc, float2 (&ra)[4], double (&rb)[2]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int e = tid + r * 256, i = e & 63, kk = e >> 6, gi = m0 + i, gk = k0 + kk;
    ra[r] = (gi < o.m && gk < K) ? A[gi + size_t(gk) * o.lda] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int e = tid + r * 256, kk = e & 15, j = n0 + (e >> 4), gk = k0 + kk;
    rb[r] = (j < nc && gk < K) ? x[gk + size_t(j) * o.ldx] : 0.0;
  }
}

__device__ void tile_df(const MOp& o, int tile, const double* x, double* y, int nc, unsigned char* smem) {
  float (*Ah)[GM + 1] = reinterpret_cast<float (*)[GM + 1]>(smem);
  float (*Al)[GM + 1] = Ah + 16;
  float (*Bh)[DN + 1] = reinterpret_cast<float (*)[DN + 1]>(smem + 32 * (GM + 1) * sizeof(float));
  float (*Bl)[DN + 1] = Bh + 16;
  const float2* A = static_cast<const float2*>(o.A);
  const int m0 = (tile >> 1) * GM, n0 = (tile & 1) * DN, K = o.n;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float s[4][2], c[4][2], H[4][2], L[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) s[i][j] = c[i][j] = H[i][j] = L[i][j] = 0.f;
  float2 ra[4];
  double rb[2];
  df_load(o, A, x, m0, n0, 0, K, nc, ra, rb);
  int since = 0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * 256;
      Ah[e >> 6][e & 63] = ra[r].x;
      Al[e >> 6][e & 63] = ra[r].y;
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int e = tid + r * 256;
      float h, l;
      df_split_bits(rb[r], h, l);
      Bh[e & 15][e >> 4] = h;
      Bl[e & 15][e >> 4] = l;
    }
    __syncthreads();
    if (k0 + 16 < K) df_load(o, A, x, m0, n0, k0 + 16, K, nc, ra, rb);
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      float ah[4], al[4], bh[2], bl[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) { ah[i] = Ah[kk][ty + 16 * i]; al[i] = Al[kk][ty + 16 * i]; }
#pragma unroll
      for (int j = 0; j < 2; ++j) { bh[j] = Bh[kk][tx + 16 * j]; bl[j] = Bl[kk][tx + 16 * j]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) df_mac(s[i][j], c[i][j], ah[i], al[i], bh[j], bl[j]);
    }
    if (++since == 8) {
      since = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) df_flush(H[i][j], L[i][j], s[i][j], c[i][j]);
    }
  }
  // alpha and beta are almost always +-1 / 0 / 1: tested once per tile, so
  // that the epilogue's FP64 work is one addition per output (two with beta)
  const bool a_one = o.alpha == 1.0, a_neg1 = o.alpha == -1.0, b_zero = o.beta == 0.0, b_one = o.beta == 1.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      df_flush(H[i][j], L[i][j], s[i][j], c[i][j]);
      const int gj = n0 + tx + 16 * j;
      if (gi >= o.m || gj >= nc) continue;
      double* yp = y + gi + size_t(gj) * o.ldy;
      double v = f2d_bits(H[i][j]) + f2d_bits(L[i][j]);
      if (a_neg1) v = -v;
      else if (!a_one) v *= o.alpha;
      if (b_one) v += *yp;
      else if (!b_zero) v += o.beta * *yp;
      *yp = v;
    }
  }
  __syncthreads();
}

// ---- FP32 or BF16 factors, FP32 vectors and accumulation: K in steps of 32
__device__ __forceinline__ float widen(float a) { return a; }
__device__ __forceinline__ float widen(__nv_bfloat16 a) { return __bfloat162float(a); }

template <class MT>
__device__ __forceinline__ void f32_load(const MOp& o, const MT* A, const float* x, int m0, int k0, int K, int nc,
                                         float (&ra)[8], float (&rb)[8]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int e = tid + r * 256, i = e & 63, kk = e >> 6, gi = m0 + i, gk = k0 + kk;
    ra[r] = (gi < o.m && gk < K) ? widen(A[gi + size_t(gk) * o.lda]) : 0.f;
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int e = tid + r * 256, kk = e & 31, j = e >> 5, gk = k0 + kk;
    rb[r] = (j < nc && gk < K) ? x[gk + size_t(j) * o.ldx] : 0.f;
  }
}

template <class MT>
__device__ void tile_f32(const MOp& o, int tile, const float* x, float* y, int nc, unsigned char* smem) {
  float (*As)[GM + 1] = reinterpret_cast<float (*)[GM + 1]>(smem);
  float (*Bs)[GN + 1] = As + 32;
  const MT* A = static_cast<const MT*>(o.A);
  const int m0 = tile * GM, K = o.n;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  float ra[8], rb[8];
  f32_load<MT>(o, A, x, m0, 0, K, nc, ra, rb);
  for (int k0 = 0; k0 < K; k0 += 32) {
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = tid + r * 256;
      As[e >> 6][e & 63] = ra[r];
      Bs[e & 31][e >> 5] = rb[r];
    }
    __syncthreads();
    if (k0 + 32 < K) f32_load<MT>(o, A, x, m0, k0 + 32, K, nc, ra, rb);
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + ty + 16 * i;
    if (gi >= o.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = tx + 16 * j;
      if (gj >= nc) continue;
      float* yp = y + gi + size_t(gj) * o.ldy;
      float v = float(o.alpha) * acc[i][j];
      if (o.beta != 0.0) v += float(o.beta) * *yp;
      *yp = v;
    }
  }
  __syncthreads();
}

// Tile kinds: one kernel per kind, so that each is register-allocated for
// its own arithmetic (the double-FP32 tile needs about 120 registers).
enum { TK_F64 = 0, TK_DF = 1, TK_F32 = 2 };

template <class T, int TK>
__global__ void __launch_bounds__(256, 2) k_gprogram(const MOp* __restrict__ ops, const int* __restrict__ tile0,
                                                  const int* __restrict__ top, const int* __restrict__ phase,
                                                  int nphases, GB<T> B, int c0, int nc, int* counters,
                                                  long long* ptimes) {
  cg::grid_group grid = cg::this_grid();
  if (ptimes && blockIdx.x == 0 && threadIdx.x == 0) ptimes[nphases] = clock64();
  __shared__ __align__(16) unsigned char smem[kSmem];
  __shared__ int s_next;
  for (int ph = 0; ph < nphases; ++ph) {
    const int t0 = tile0[phase[ph]], t1 = tile0[phase[ph + 1]];
    // tiles are taken from a per-phase counter (longest first, by the host's
    // ordering), so a CTA that finishes early takes the next tile
    for (;;) {
      if (threadIdx.x == 0) s_next = t0 + atomicAdd(counters + ph, 1);
      __syncthreads();
      const int t = s_next;
      __syncthreads();
      if (t >= t1) break;
      const int oi = top[t];
      const MOp& o = ops[oi];
      const int tile = t - tile0[oi];
      if (o.kind == MOP_GEMM) {
        const T* x = B.p[o.xb] + o.xo + size_t(c0) * o.ldx;
        T* y = B.p[o.yb] + o.yo + size_t(c0) * o.ldy;
        if constexpr (TK == TK_F64) tile_f64(o, tile, x, y, nc, smem);
        else if constexpr (TK == TK_DF) tile_df(o, tile, x, y, nc, smem);
        else {
          if (o.atype == MA_BF16) tile_f32<__nv_bfloat16>(o, tile, x, y, nc, smem);
          else tile_f32<float>(o, tile, x, y, nc, smem);
        }
      } else {
        // one thread per (entry, right-hand side), entries fastest
        const int idx = tile * TE + threadIdx.x, i = idx % o.m, r = idx / o.m;
        if (r < nc) {
          const T* x = (o.kind == MOP_ZERO) ? nullptr : B.p[o.xb] + o.xo + size_t(c0) * o.ldx;
          T* y = B.p[o.yb] + o.yo + size_t(c0) * o.ldy;
          if (o.kind == MOP_COPY) {
            y[(o.iy ? o.iy[i] : i) + size_t(r) * o.ldy] = x[(o.ix ? o.ix[i] : i) + size_t(r) * o.ldx];
          } else if (o.kind == MOP_ZERO) {
            y[(o.iy ? o.iy[i] : i) + size_t(r) * o.ldy] = T(0);
          } else {
            // REDUCE: parts are m apart in x; four interleaved chains, added
            // in a fixed order
            const T* xr = x + i + size_t(r) * o.ldx;
            T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
            int q = 0;
            for (; q + 3 < o.n; q += 4) {
              s0 += xr[size_t(q) * o.m];
              s1 += xr[size_t(q + 1) * o.m];
              s2 += xr[size_t(q + 2) * o.m];
              s3 += xr[size_t(q + 3) * o.m];
            }
            for (; q < o.n; ++q) s0 += xr[size_t(q) * o.m];
            T* yp = y + i + size_t(r) * o.ldy;
            T v = T(o.alpha) * ((s0 + s1) + (s2 + s3));
            if (o.beta != 0.0) v += T(o.beta) * *yp;
            *yp = v;
          }
        }
      }
    }
    grid.sync();
    if (ptimes && blockIdx.x == 0 && threadIdx.x == 0) ptimes[ph] = clock64();
  }
}

template <class T>
const void* gkernel(int tk) {
  if constexpr (std::is_same<T, double>::value)
    return tk == TK_DF ? reinterpret_cast<const void*>(&k_gprogram<double, TK_DF>)
                       : reinterpret_cast<const void*>(&k_gprogram<double, TK_F64>);
  else
    return reinterpret_cast<const void*>(&k_gprogram<float, TK_F32>);
}

int op_tiles(const MOp& o, int tk) {
  return o.kind == MOP_GEMM ? (o.m + GM - 1) / GM * (tk == TK_DF ? GN / DN : 1)
                            : int((static_cast<long long>(o.m) * GN + TE - 1) / TE);
}

std::vector<MOp>& phase_at(std::vector<std::vector<MOp>>& ph, int p) {
  if (int(ph.size()) <= p) ph.resize(p + 1);
  return ph[p];
}

}  // namespace

// RW_GPROG_TIMES=1 (diagnostics): print each phase's tiles and cycles (as
// seen by CTA 0) after every run; synchronises the stream
static bool gphase_times() {
  static const bool on = [] {
    const char* e = std::getenv("RW_GPROG_TIMES");
    return e && e[0] == '1';
  }();
  return on;
}

template <class T>
void GProgram<T>::add_gemm(int p, const void* A, int atype, int m, int n, int lda, int xb, long long xo, int ldx,
                           int yb, long long yo, int ldy, double alpha, double beta) {
  if (m <= 0) return;
  if (std::is_same<T, double>::value)
    require(atype == MA_F64 || atype == MA_DF, "GEMM program: FP64 vectors take FP64 or double-FP32 factors");
  else
    require(atype == MA_F32 || atype == MA_BF16, "GEMM program: FP32 vectors take FP32 or BF16 factors");
  const int tk = atype == MA_DF ? TK_DF : atype == MA_F64 ? TK_F64 : TK_F32;
  require(tk_ < 0 || tk_ == tk, "GEMM program: FP64 and double-FP32 factors cannot share a program");
  tk_ = tk;
  if (atype == MA_DF) prof_class_df_ = true;
  MOp o{};
  o.kind = MOP_GEMM;
  o.m = m; o.n = n; o.A = A; o.lda = lda; o.atype = atype;
  o.xb = xb; o.xo = xo; o.ldx = ldx; o.yb = yb; o.yo = yo; o.ldy = ldy;
  o.alpha = alpha; o.beta = beta;
  phase_at(phases_, p).push_back(o);
  flops_ += 2.0 * double(m) * double(n);
}

template <class T>
void GProgram<T>::copy(int p, int n, int xb, long long xo, int ldx, const int* ix, int yb, long long yo, int ldy,
                       const int* iy) {
  if (n <= 0) return;
  MOp o{};
  o.kind = MOP_COPY;
  o.m = n; o.xb = xb; o.xo = xo; o.ldx = ldx; o.ix = ix; o.yb = yb; o.yo = yo; o.ldy = ldy; o.iy = iy;
  phase_at(phases_, p).push_back(o);
}

template <class T>
void GProgram<T>::zero(int p, int n, int yb, long long yo, int ldy, const int* iy) {
  if (n <= 0) return;
  MOp o{};
  o.kind = MOP_ZERO;
  o.m = n; o.yb = yb; o.yo = yo; o.ldy = ldy; o.iy = iy;
  phase_at(phases_, p).push_back(o);
}

template <class T>
long long GProgram<T>::ws_alloc(long long elems) {
  const long long o = ws_;
  ws_ += (elems + 31) / 32 * 32;
  return o;
}

template <class T>
void GProgram<T>::finalize(cudaStream_t s_caller, cudaStream_t alloc) {
  // uploads on the allocation stream when there is one (the memory is
  // ordered there), synchronised before returning
  AllocStreamScope scope(alloc);
  cudaStream_t s = alloc ? alloc : s_caller;
  int dev = 0, nsm = 0;
  RW_CUDA(cudaGetDevice(&dev));
  RW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // A tile walks its product's whole inner dimension on one SM, and a
  // 64 x 64 x 16 step is 65536 multiply-adds (~16 us of one SM's FP64 pipe,
  // ~3 us in double-FP32): inner dimensions beyond a per-kind limit are cut
  // into chunks of at most that limit, and in a phase with fewer tiles than two per SM into chunks
  // of at least 32 until the phase has about two tiles per SM.  The partial
  // products go to the workspace and a reduce op in an extra phase adds them
  // in a fixed order.
  std::vector<std::vector<MOp>> out;
  for (auto& ph : phases_) {
    int tiles = 0;
    for (const MOp& o : ph) tiles += op_tiles(o, tk_);
    const bool thin = tiles < 2 * nsm;
    std::vector<MOp> cur, red;
    for (const MOp& o : ph) {
      int parts = 1;
      if (o.kind == MOP_GEMM) {
        if (thin && o.n >= 64) parts = std::min((o.n + 31) / 32, std::max(1, (2 * nsm) / std::max(tiles, 1)));
        const int kmax = tk_ == TK_F64 ? KMAX_F64 : tk_ == TK_DF ? KMAX_DF : KMAX_F32;
        parts = std::max(parts, (o.n + kmax - 1) / kmax);
      }
      if (parts <= 1) {
        cur.push_back(o);
        continue;
      }
      const int chunk = ((o.n + parts - 1) / parts + 31) / 32 * 32;
      parts = (o.n + chunk - 1) / chunk;
      const long long pw = ws_alloc((long long)parts * o.m);
      const size_t esz = o.atype == MA_F64 ? 8 : o.atype == MA_DF ? 8 : o.atype == MA_F32 ? 4 : 2;
      for (int q = 0; q < parts; ++q) {
        MOp g = o;
        const int k0 = q * chunk, k1 = std::min(o.n, k0 + chunk);
        g.A = static_cast<const char*>(o.A) + size_t(k0) * o.lda * esz;
        g.n = k1 - k0;
        g.xo = o.xo + k0;
        g.yb = wsb_; g.yo = pw + (long long)q * o.m; g.ldy = -1;
        g.alpha = 1.0; g.beta = 0.0;
        cur.push_back(g);
      }
      MOp r{};
      r.kind = MOP_REDUCE;
      r.m = o.m; r.n = parts;
      r.xb = wsb_; r.xo = pw; r.ldx = -1;
      r.yb = o.yb; r.yo = o.yo; r.ldy = o.ldy;
      r.alpha = o.alpha; r.beta = o.beta;
      red.push_back(r);
    }
    out.push_back(cur);
    if (!red.empty()) out.push_back(red);
  }
  for (auto& ph : out)
    for (MOp& o : ph) {
      if (o.ldx == -1) o.ldx = int(ws_);
      if (o.ldy == -1) o.ldy = int(ws_);
    }
  // within a phase the longest tiles go first (inner dimension for
  // products, parts for reduces), so the dynamic tile counter balances the SMs
  for (auto& ph : out)
    std::stable_sort(ph.begin(), ph.end(), [](const MOp& a, const MOp& b) {
      auto cost = [](const MOp& o) { return o.kind == MOP_GEMM ? o.n : o.kind == MOP_REDUCE ? o.n / 8 : 0; };
      return cost(a) > cost(b);
    });
  std::vector<MOp> flat;
  std::vector<int> phase(1, 0), tile0(1, 0);
  int maxt = 1;
  for (auto& ph : out) {
    int tph = 0;
    for (const MOp& o : ph) {
      flat.push_back(o);
      tile0.push_back(tile0.back() + op_tiles(o, tk_));
      tph += op_tiles(o, tk_);
    }
    phase.push_back(int(flat.size()));
    maxt = std::max(maxt, tph);
  }
  std::vector<int> top(std::max(tile0.back(), 1), 0);
  for (size_t q = 0; q + 1 < tile0.size(); ++q)
    for (int t = tile0[q]; t < tile0[q + 1]; ++t) top[t] = int(q);
  nph_ = int(out.size());
  ph_tiles_.clear();
  ph_mac_.clear();
  ph_kmax_.clear();
  for (auto& q : out) {
    int tq = 0, km = 0;
    double mac = 0.0;
    for (const MOp& o : q) {
      tq += op_tiles(o, tk_);
      if (o.kind == MOP_GEMM) { mac += double(o.m) * o.n; km = std::max(km, o.n); }
    }
    ph_tiles_.push_back(tq);
    ph_mac_.push_back(mac);
    ph_kmax_.push_back(km);
  }
  d_ops_ = to_device(flat.empty() ? std::vector<MOp>(1) : flat, s);
  d_phase_ = to_device(phase, s);
  d_tile0_ = to_device(tile0, s);
  d_top_ = to_device(top, s);
  int per = 0;
  RW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gkernel<T>(tk_), 256, 0));
  grid_ = std::max(1, std::min(maxt, nsm * std::max(per, 1)));
  RW_CUDA(cudaStreamSynchronize(s));
  done_ = true;
}

template <class T>
void GProgram<T>::run(T* const* bases, int nrhs, cudaStream_t s) const {
  require(done_, "GEMM program used before finalize");
  if (nph_ == 0 || nrhs <= 0) return;
  GB<T> B;
  for (int i = 0; i < kGBases; ++i) B.p[i] = bases[i];
  const MOp* ops = d_ops_.p;
  const int* t0 = d_tile0_.p;
  const int* top = d_top_.p;
  const int* ph = d_phase_.p;
  int nphases = nph_;
  // profiler class: the program's arithmetic decides which peak applies
  int cls = KC_GEMM;
  if (!std::is_same<T, double>::value) cls = KC_GEMM_F32;
  else if (prof_class_df_) cls = KC_GEMM_DF;
  for (int c0 = 0; c0 < nrhs; c0 += GN) {
    int nc = std::min(GN, nrhs - c0);
    TBuf<long long> times(gphase_times() ? size_t(nph_ + 1) : 0, s);
    long long* pt = times.p;
    TBuf<int> ctr(size_t(nph_), s);
    RW_CUDA(cudaMemsetAsync(ctr.p, 0, size_t(nph_) * sizeof(int), s));
    int* cp = ctr.p;
    void* args[] = {(void*)&ops, (void*)&t0, (void*)&top, (void*)&ph, (void*)&nphases, (void*)&B, (void*)&c0,
                    (void*)&nc, (void*)&cp, (void*)&pt};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ProfScope prof(cls, s, flops_ * nc, 0.0);
    RW_CUDA(cudaLaunchKernelExC(&cfg, gkernel<T>(tk_), args));
    RW_CHECK_LAUNCH();
    if (gphase_times()) {
      std::vector<long long> h(nph_ + 1);
      RW_CUDA(cudaMemcpyAsync(h.data(), times.p, h.size() * sizeof(long long), cudaMemcpyDeviceToHost, s));
      RW_CUDA(cudaStreamSynchronize(s));
      std::fprintf(stderr, "[rw gprogram] kind %d, %d phases, grid %d, %d right-hand sides:\n", tk_, nph_, grid_, nc);
      long long prev = h[nph_];
      for (int q = 0; q < nph_; ++q) {
        std::fprintf(stderr, "[rw gprogram]   phase %2d: %5d tiles, K <= %5d, %9.3f M multiply-adds, %8lld cycles\n", q,
                     ph_tiles_[q], ph_kmax_[q], 1e-6 * ph_mac_[q] * nc, h[q] - prev);
        prev = h[q];
      }
    }
  }
}

template class GProgram<double>;
template class GProgram<float>;

}  // namespace rw
