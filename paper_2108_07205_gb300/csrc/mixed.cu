// Batched GEMMs of the mixed-precision path (Sec. 4.2):
//  * FP32 accumulation (FP32 or BF16 matrices, FP32 vectors): the HBS inverse
//    sweeps and the Woodbury correction of the low-precision preconditioner
//    once many right-hand sides make them matrix-matrix products;
//  * double-FP32: the operator products of the FGMRES residual, with each FP64
//    factor held as an FP32 pair and every product and sum compensated, so
//    that the residual keeps FP64-level accuracy while the work runs on the
//    FP32 units (on this part 64 FP32 lanes per FP64 lane).
// Both follow batched_gemm (dense.cu): 64 x 64 output tiles, one problem list
// per launch, split-K with partial sums added in a fixed order when the tiles
// cannot fill the GPU.
#include "dense.cuh"
#include "dfarith.cuh"
#include <algorithm>
#include <cmath>

namespace rw {

namespace {

int device_sms() {
  static int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 152;
    }
    return v;
  }();
  return n;
}

__device__ __forceinline__ int find_prob(const int* offs, int nprob, int tile) {
  int lo = 0, hi = nprob;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (offs[mid] <= tile) lo = mid; else hi = mid;
  }
  return lo;
}

// Split-K plan shared by both GEMMs: chunks in proportion to each problem's
// share of the work when the output tiles cannot give three CTAs per SM.
template <class W>
long long plan_split(std::vector<W>& ws, std::vector<int>& offs, int kstep) {
  long long tiles_all = 0;
  for (auto& w : ws) tiles_all += (long long)w.tilesM * w.tilesN;
  const long long target = 3LL * device_sms();
  double tile_k = 0.0;
  for (auto& w : ws) tile_k += double(w.tilesM) * w.tilesN * std::max(w.p.k, 1);
  const double per_cta = tile_k / double(target);
  long long scratch = 0;
  offs.assign(1, 0);
  for (auto& w : ws) {
    const long long tiles = (long long)w.tilesM * w.tilesN;
    w.nsplit = 1;
    w.kchunk = std::max(w.p.k, 1);
    w.scratch_off = 0;
    if (tiles_all < target && w.p.k >= 128) {
      int ns = int(std::min<double>(std::ceil(double(w.p.k) / std::max(per_cta, 1.0)), double(w.p.k / 64)));
      ns = std::min(ns, 128);
      if (ns > 1) {
        w.kchunk = ((w.p.k + ns - 1) / ns + kstep - 1) / kstep * kstep;
        w.nsplit = (w.p.k + w.kchunk - 1) / w.kchunk;
        w.scratch_off = scratch;
        scratch += (long long)w.nsplit * w.p.m * w.p.n;
      }
    }
    offs.push_back(offs.back() + int(tiles * w.nsplit));
  }
  return scratch;
}

// ------------------------------------------------------------------ FP32
constexpr int FM = 64, FN = 64, FK = 32;

template <class MT>
struct GemmF32Work {
  GemmF32Prob<MT> p;
  int tilesM, tilesN, nsplit, kchunk;
  long long scratch_off;
};

__device__ __forceinline__ float widen(float a) { return a; }
__device__ __forceinline__ float widen(__nv_bfloat16 a) { return __bfloat162float(a); }

template <class MT>
__global__ void __launch_bounds__(256) k_gemm_f32(const GemmF32Work<MT>* work, const int* offs, int nprob,
                                                  float* scratch) {
  __shared__ float As[FK][FM + 1];
  __shared__ float Bs[FK][FN + 1];
  const int tile = blockIdx.x;
  const int b = find_prob(offs, nprob, tile);
  const GemmF32Work<MT> Wk = work[b];
  const GemmF32Prob<MT>& P = Wk.p;
  const int tilesMN = Wk.tilesM * Wk.tilesN;
  const int t = tile - offs[b];
  const int split = t / tilesMN, tt = t % tilesMN;
  const int m0 = (tt % Wk.tilesM) * FM, n0 = (tt / Wk.tilesM) * FN;
  const int kb = split * Wk.kchunk, ke = min(P.k, kb + Wk.kchunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += FK) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = tid + r * 256;  // 0..2047
      const int i = e & 63, kk = e >> 6;
      const int gi = m0 + i, gk = k0 + kk;
      As[kk][i] = (gi < P.m && gk < ke) ? widen(P.A[gi + size_t(gk) * P.lda]) : 0.f;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = tid + r * 256;
      const int kk = e & 31, j = e >> 5;
      const int gj = n0 + j, gk = k0 + kk;
      Bs[kk][j] = (gj < P.n && gk < ke) ? P.B[gk + size_t(gj) * P.ldb] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < FK; ++kk) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + ty + 16 * i;
    if (gi >= P.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = n0 + tx + 16 * j;
      if (gj >= P.n) continue;
      if (Wk.nsplit > 1) {
        scratch[Wk.scratch_off + (size_t(split) * P.n + gj) * P.m + gi] = acc[i][j];
      } else {
        float* c = P.C + gi + size_t(gj) * P.ldc;
        float v = P.alpha * acc[i][j];
        if (P.beta != 0.f) v += P.beta * *c;
        *c = v;
      }
    }
  }
}

template <class MT>
__global__ void k_gemm_f32_reduce(const GemmF32Work<MT>* work, const float* scratch) {
  const GemmF32Work<MT> Wk = work[blockIdx.y];
  if (Wk.nsplit <= 1) return;
  const GemmF32Prob<MT>& P = Wk.p;
  for (int j = blockIdx.x; j < P.n; j += gridDim.x)
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) {
      float s = 0.f;
      for (int q = 0; q < Wk.nsplit; ++q) s += scratch[Wk.scratch_off + (size_t(q) * P.n + j) * P.m + i];
      float* c = P.C + i + size_t(j) * P.ldc;
      float v = P.alpha * s;
      if (P.beta != 0.f) v += P.beta * *c;
      *c = v;
    }
}

// ------------------------------------------------------------------ double-FP32
constexpr int DM = 64, DN = 64, DK = 16, DFLUSH = 8;  // flush every DFLUSH * DK = 128 terms

struct GemmDfWork {
  GemmDfProb p;
  int tilesM, tilesN, nsplit, kchunk;
  long long scratch_off;
};

__global__ void __launch_bounds__(256) k_gemm_df(const GemmDfWork* work, const int* offs, int nprob,
                                                 double* scratch) {
  __shared__ float Ah[DK][DM + 1], Al[DK][DM + 1];
  __shared__ float Bh[DK][DN + 1], Bl[DK][DN + 1];
  const int tile = blockIdx.x;
  const int b = find_prob(offs, nprob, tile);
  const GemmDfWork Wk = work[b];
  const GemmDfProb& P = Wk.p;
  const int tilesMN = Wk.tilesM * Wk.tilesN;
  const int t = tile - offs[b];
  const int split = t / tilesMN, tt = t % tilesMN;
  const int m0 = (tt % Wk.tilesM) * DM, n0 = (tt / Wk.tilesM) * DN;
  const int kb = split * Wk.kchunk, ke = min(P.k, kb + Wk.kchunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float s[4][4], c[4][4], H[4][4], L[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s[i][j] = c[i][j] = H[i][j] = L[i][j] = 0.f;
  int since = 0;
  for (int k0 = kb; k0 < ke; k0 += DK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * 256;  // 0..1023
      const int i = e & 63, kk = e >> 6;
      const int gi = m0 + i, gk = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (gi < P.m && gk < ke) v = P.A[gi + size_t(gk) * P.lda];
      Ah[kk][i] = v.x;
      Al[kk][i] = v.y;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * 256;
      const int kk = e & 15, j = e >> 4;
      const int gj = n0 + j, gk = k0 + kk;
      float h = 0.f, l = 0.f;
      if (gj < P.n && gk < ke) {
        df_split_bits(P.B[gk + size_t(gj) * P.ldb], h, l);
      }
      Bh[kk][j] = h;
      Bl[kk][j] = l;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < DK; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { ah[i] = Ah[kk][ty + 16 * i]; al[i] = Al[kk][ty + 16 * i]; }
#pragma unroll
      for (int j = 0; j < 4; ++j) { bh[j] = Bh[kk][tx + 16 * j]; bl[j] = Bl[kk][tx + 16 * j]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_mac(s[i][j], c[i][j], ah[i], al[i], bh[j], bl[j]);
    }
    __syncthreads();
    if (++since == DFLUSH) {
      since = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_flush(H[i][j], L[i][j], s[i][j], c[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) df_flush(H[i][j], L[i][j], s[i][j], c[i][j]);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + ty + 16 * i;
    if (gi >= P.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = n0 + tx + 16 * j;
      if (gj >= P.n) continue;
      const double v = f2d_bits(H[i][j]) + f2d_bits(L[i][j]);
      if (Wk.nsplit > 1) {
        scratch[Wk.scratch_off + (size_t(split) * P.n + gj) * P.m + gi] = v;
      } else {
        double* cp = P.C + gi + size_t(gj) * P.ldc;
        double o = P.alpha * v;
        if (P.beta != 0.0) o += P.beta * *cp;
        *cp = o;
      }
    }
  }
}

__global__ void k_gemm_df_reduce(const GemmDfWork* work, const double* scratch) {
  const GemmDfWork Wk = work[blockIdx.y];
  if (Wk.nsplit <= 1) return;
  const GemmDfProb& P = Wk.p;
  for (int j = blockIdx.x; j < P.n; j += gridDim.x)
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) {
      double v = 0.0;
      for (int q = 0; q < Wk.nsplit; ++q) v += scratch[Wk.scratch_off + (size_t(q) * P.n + j) * P.m + i];
      double* cp = P.C + i + size_t(j) * P.ldc;
      double o = P.alpha * v;
      if (P.beta != 0.0) o += P.beta * *cp;
      *cp = o;
    }
}

__global__ void k_d2df(const double* in, float2* out, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const double v = in[i];
    const float h = __double2float_rn(v);
    out[i] = make_float2(h, __double2float_rn(v - double(h)));
  }
}

}  // namespace

template <class MT>
void batched_gemm_f32(const std::vector<GemmF32Prob<MT>>& probs, cudaStream_t s) {
  std::vector<GemmF32Work<MT>> ws;
  for (const auto& p : probs) {
    if (p.m <= 0 || p.n <= 0) continue;
    GemmF32Work<MT> w{};
    w.p = p;
    w.tilesM = ceil_div(p.m, FM);
    w.tilesN = ceil_div(p.n, FN);
    ws.push_back(w);
  }
  if (ws.empty()) return;
  std::vector<int> offs;
  const long long scratch = plan_split(ws, offs, FK);
  TBuf<float> sc(size_t(scratch), s);
  auto dw = to_device_tmp(ws, s);
  auto doff = to_device_tmp(offs, s);
  double fl = 0.0, by = 0.0;
  for (auto& w : ws) {
    fl += 2.0 * w.p.m * w.p.n * double(w.p.k);
    by += double(sizeof(MT)) * w.p.m * double(w.p.k) + 4.0 * (double(w.p.k) * w.p.n + 2.0 * w.p.m * w.p.n);
  }
  ProfScope ps(KC_GEMM_F32, s, fl, by);
  k_gemm_f32<MT><<<offs.back(), 256, 0, s>>>(dw.p, doff.p, int(ws.size()), sc.p);
  RW_CHECK_LAUNCH();
  if (scratch) {
    int mn = 0;
    for (auto& w : ws) mn = std::max(mn, w.p.n);
    k_gemm_f32_reduce<MT><<<dim3(std::min(mn, 1024), int(ws.size())), 256, 0, s>>>(dw.p, sc.p);
    RW_CHECK_LAUNCH();
  }
}
template void batched_gemm_f32<float>(const std::vector<GemmF32Prob<float>>&, cudaStream_t);
template void batched_gemm_f32<__nv_bfloat16>(const std::vector<GemmF32Prob<__nv_bfloat16>>&, cudaStream_t);

void batched_gemm_df(const std::vector<GemmDfProb>& probs, cudaStream_t s) {
  std::vector<GemmDfWork> ws;
  for (const auto& p : probs) {
    if (p.m <= 0 || p.n <= 0) continue;
    GemmDfWork w{};
    w.p = p;
    w.tilesM = ceil_div(p.m, DM);
    w.tilesN = ceil_div(p.n, DN);
    ws.push_back(w);
  }
  if (ws.empty()) return;
  std::vector<int> offs;
  const long long scratch = plan_split(ws, offs, DK * DFLUSH);
  TBuf<double> sc(size_t(scratch), s);
  auto dw = to_device_tmp(ws, s);
  auto doff = to_device_tmp(offs, s);
  double fl = 0.0, by = 0.0;
  for (auto& w : ws) {
    fl += 2.0 * w.p.m * w.p.n * double(w.p.k);
    by += 8.0 * (double(w.p.m) * w.p.k + double(w.p.k) * w.p.n + 2.0 * w.p.m * w.p.n);
  }
  ProfScope ps(KC_GEMM_DF, s, fl, by);
  k_gemm_df<<<offs.back(), 256, 0, s>>>(dw.p, doff.p, int(ws.size()), sc.p);
  RW_CHECK_LAUNCH();
  if (scratch) {
    int mn = 0;
    for (auto& w : ws) mn = std::max(mn, w.p.n);
    k_gemm_df_reduce<<<dim3(std::min(mn, 1024), int(ws.size())), 256, 0, s>>>(dw.p, sc.p);
    RW_CHECK_LAUNCH();
  }
}

void copy_d2df(const double* in, float2* out, size_t n, cudaStream_t s) {
  if (!n) return;
  const int grid = int(std::min<size_t>((n + 255) / 256, size_t(16) * device_sms()));
  k_d2df<<<grid, 256, 0, s>>>(in, out, n);
  RW_CHECK_LAUNCH();
}

// matvec for many right-hand sides in the low-precision types: GEMV chunks of
// at most 8 columns up to 8, the FP32-accumulation GEMM above that.
template <class MT>
static void matvec_lowp(const std::vector<GemvProb<float, MT>>& probs, int nrhs, cudaStream_t s) {
  if (probs.empty() || nrhs <= 0) return;
  if (nrhs <= 8) {
    size_t sc = gemv_scratch_elems(probs, nrhs);
    TBuf<float> scratch(sc, s);
    batched_gemv(probs, nrhs, scratch.p, s);
    return;
  }
  std::vector<GemmF32Prob<MT>> g;
  for (auto& p : probs)
    g.push_back(GemmF32Prob<MT>{p.A, p.x, p.y, p.m, nrhs, p.n, p.lda, p.ldx, p.ldy, float(p.alpha), float(p.beta)});
  batched_gemm_f32(g, s);
}

template <>
void matvec<float, float>(const std::vector<GemvProb<float>>& probs, int nrhs, cudaStream_t s) {
  matvec_lowp(probs, nrhs, s);
}

template <>
void matvec<float, __nv_bfloat16>(const std::vector<GemvProb<float, __nv_bfloat16>>& probs, int nrhs,
                                  cudaStream_t s) {
  matvec_lowp(probs, nrhs, s);
}

// Double-FP32 operator products (any nrhs: the GEMM tiles are used even for a
// single column).
template <>
void matvec<double, float2>(const std::vector<GemvProb<double, float2>>& probs, int nrhs, cudaStream_t s) {
  if (probs.empty() || nrhs <= 0) return;
  std::vector<GemmDfProb> g;
  for (auto& p : probs) g.push_back(GemmDfProb{p.A, p.x, p.y, p.m, nrhs, p.n, p.lda, p.ldx, p.ldy, p.alpha, p.beta});
  batched_gemm_df(g, s);
}

}  // namespace rw
