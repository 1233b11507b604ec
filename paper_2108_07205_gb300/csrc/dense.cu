// Batched dense kernels: tiled GEMM, small-RHS GEMV with deterministic
// split-K, Gauss-Jordan inverse, column-pivoted QR interpolative
// decomposition, and fills.  One launch per problem list; each CTA finds its
// problem from a prefix sum of per-problem tile counts.
#include "dense.cuh"
#include <algorithm>
#include <cmath>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

#include <atomic>
#include <chrono>
#include <mutex>
#include <cstdlib>

namespace rw {

std::atomic<unsigned long long> g_launches{0};
thread_local cudaStream_t tl_alloc_stream = nullptr;

void pool_retain_once() {
  constexpr int kMaxDev = 64;
  static std::atomic<bool> done[kMaxDev];
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) { cudaGetLastError(); return; }
  if (done[dev].load(std::memory_order_acquire)) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev].load(std::memory_order_relaxed)) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    unsigned long long keep = 0;
    if (const char* e = std::getenv("RW_POOL_RETAIN_BYTES")) {
      keep = std::strtoull(e, nullptr, 10);
    } else {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) keep = tot / 4;
    }
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();  // a refusal leaves the default behaviour
  done[dev].store(true, std::memory_order_release);
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

Trace::Trace(cudaStream_t st, const char* w) : s(st), what(w) {
  const char* e = std::getenv("RW_TRACE");
  on = e && e[0] == '1';
  if (on) { cudaStreamSynchronize(s); t0 = now_s(); }
}

namespace {
constexpr int kSideStreams = 7;
struct SidePool {
  int dev = -1;
  cudaStream_t st[kSideStreams] = {};
  cudaEvent_t ev[kSideStreams + 1] = {};
};
thread_local SidePool tl_side;
SidePool& side_pool() {
  int dev = 0;
  RW_CUDA(cudaGetDevice(&dev));
  if (tl_side.dev != dev) {  // a thread that moved to another device starts a new pool
    tl_side = SidePool();
    tl_side.dev = dev;
  }
  return tl_side;
}
cudaEvent_t pool_event(SidePool& p, int i) {
  if (!p.ev[i]) RW_CUDA(cudaEventCreateWithFlags(&p.ev[i], cudaEventDisableTiming));
  return p.ev[i];
}
}  // namespace

ForkJoin::ForkJoin(cudaStream_t s, int n) : s_(s), n_(std::min(n, kSideStreams + 1)) {
  if (n_ > 1) RW_CUDA(cudaEventRecord(pool_event(side_pool(), 0), s_));
}

cudaStream_t ForkJoin::next() {
  if (n_ <= 1 || used_ == 0 || used_ >= n_) {
    if (used_ < n_) ++used_;
    return s_;
  }
  SidePool& p = side_pool();
  cudaStream_t& t = p.st[used_ - 1];
  if (!t) RW_CUDA(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
  RW_CUDA(cudaStreamWaitEvent(t, pool_event(p, 0), 0));
  ++used_;
  return t;
}

void ForkJoin::join() {
  if (joined_) return;
  joined_ = true;
  if (n_ <= 1) return;
  SidePool& p = side_pool();
  for (int i = 1; i < used_; ++i) {
    cudaEvent_t e = pool_event(p, i);
    RW_CUDA(cudaEventRecord(e, p.st[i - 1]));
    RW_CUDA(cudaStreamWaitEvent(s_, e, 0));
  }
}

ForkJoin::~ForkJoin() {
  if (joined_ || n_ <= 1) return;
  // best effort on an exceptional exit: keep s ordered after the side work
  SidePool& p = tl_side;
  for (int i = 1; i < used_; ++i)
    if (p.st[i - 1] && p.ev[i] && cudaEventRecord(p.ev[i], p.st[i - 1]) == cudaSuccess)
      cudaStreamWaitEvent(s_, p.ev[i], 0);
}

void Trace::mark(const char* phase) {
  if (!on) return;
  cudaStreamSynchronize(s);
  const double t = now_s();
  std::fprintf(stderr, "[rw trace] %s %-28s %8.3f ms\n", what, phase, 1e3 * (t - t0));
  t0 = t;
}

// ------------------------------------------------------------------ profiler
namespace {
struct ProfRec { cudaEvent_t a, b; int cls; double flops, bytes; };
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof;
std::atomic<bool> g_prof_on{false};
__device__ double g_id_flops;
}  // namespace

bool prof_enabled() { return g_prof_on.load(std::memory_order_relaxed); }

double* id_flops_counter() {
  if (!prof_enabled()) return nullptr;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_id_flops) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return static_cast<double*>(p);
}

ProfScope::ProfScope(int cls_, cudaStream_t st, double fl, double by)
    : on(prof_enabled()), cls(cls_), s(st), flops(fl), bytes(by) {
  if (!on) return;
  cudaEventCreate(&a);
  cudaEventRecord(a, s);
}

ProfScope::~ProfScope() {
  if (!on) return;
  cudaEvent_t b;
  cudaEventCreate(&b);
  cudaEventRecord(b, s);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.push_back(ProfRec{a, b, cls, flops, bytes});
}

void profile_enable(bool on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaDeviceSynchronize();
  for (auto& r : g_prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  g_prof.clear();
  double z = 0.0;
  cudaMemcpyToSymbol(g_id_flops, &z, sizeof(double));
  g_prof_on.store(on);
}

void profile_read(long long* launches, double* ms, double* flops, double* bytes) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaDeviceSynchronize();
  for (int c = 0; c < KC_COUNT; ++c) { launches[c] = 0; ms[c] = 0; flops[c] = 0; bytes[c] = 0; }
  for (auto& r : g_prof) {
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    launches[r.cls] += 1;
    ms[r.cls] += t;
    flops[r.cls] += r.flops;
    bytes[r.cls] += r.bytes;
  }
  double idf = 0.0;
  cudaMemcpyFromSymbol(&idf, g_id_flops, sizeof(double));
  flops[KC_ID] += idf;
}

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

struct GemmWork {
  GemmProb p;
  int tilesM, tilesN, nsplit, kchunk;
  long long scratch_off;  // partial sums (nsplit x m x n) when nsplit > 1
};

__global__ void __launch_bounds__(256) k_gemm(const GemmWork* work, const int* offs, int nprob, double* scratch) {
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  const int tile = blockIdx.x;
  const int b = find_problem(offs, nprob, tile);
  const GemmWork Wk = work[b];
  const GemmProb& P = Wk.p;
  const int tilesM = Wk.tilesM, tilesMN = Wk.tilesM * Wk.tilesN;
  const int t = tile - offs[b];
  const int split = t / tilesMN, tt = t % tilesMN;
  const int m0 = (tt % tilesM) * GBM, n0 = (tt / tilesM) * GBN;
  const int kb = split * Wk.kchunk, ke = min(P.k, kb + Wk.kchunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = kb; k0 < ke; k0 += GBK) {
    // load op(A)[m0 : m0+64, k0 : k0+16]
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * 256;  // 0..1023
      int i, kk;
      if (!P.ta) { i = e & 63; kk = e >> 6; } else { kk = e & 15; i = e >> 4; }
      int gi = m0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < P.m && gk < ke)
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
      if (gj < P.n && gk < ke)
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
      if (Wk.nsplit > 1) {
        scratch[Wk.scratch_off + (size_t(split) * P.n + gj) * P.m + gi] = acc[i][j];
      } else {
        double* c = P.C + gi + size_t(gj) * P.ldc;
        double v = P.alpha * acc[i][j];
        if (P.beta != 0.0) v += P.beta * *c;
        *c = v;
      }
    }
  }
}

// C = alpha * sum_s partial_s + beta C for split problems (fixed order).
__global__ void k_gemm_reduce(const GemmWork* work, const double* scratch) {
  const GemmWork Wk = work[blockIdx.y];
  if (Wk.nsplit <= 1) return;
  const GemmProb& P = Wk.p;
  for (int j = blockIdx.x; j < P.n; j += gridDim.x)
  for (int i = threadIdx.x; i < P.m; i += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < Wk.nsplit; ++q) s += scratch[Wk.scratch_off + (size_t(q) * P.n + j) * P.m + i];
    double* c = P.C + i + size_t(j) * P.ldc;
    double v = P.alpha * s;
    if (P.beta != 0.0) v += P.beta * *c;
    *c = v;
  }
}

// ------------------------------------------------------------------ GEMV
// Tile = 64 rows x one column chunk; 256 threads = 64 rows x 4 column lanes.
constexpr int VR = 64;
constexpr int VCHUNK = 2048;  // columns per split-K chunk

template <class T, class MT = T>
struct GemvWork {  // device-side descriptor (adds split-K bookkeeping)
  GemvProb<T, MT> p;
  int tilesM, nchunk;
  long long scratch_off;  // offset of this problem's partials (elements)
};

template <class T> struct Acc { typedef double type; };
template <> struct Acc<float> { typedef float type; };

template <class T, class MT, int NR>
__global__ void __launch_bounds__(256) k_gemv(const GemvWork<T, MT>* work, const int* offs, int nprob,
                                              T* scratch) {
  typedef typename Acc<T>::type A_t;
  const int tile = blockIdx.x;
  const int b = find_problem(offs, nprob, tile);
  const GemvWork<T, MT> W = work[b];
  const GemvProb<T, MT>& P = W.p;
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
      const MT* a = P.A + row + size_t(cb) * P.lda;
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

template <class T, class MT, int NR>
__global__ void k_gemv_reduce(const GemvWork<T, MT>* work, int nprob, const T* scratch) {
  typedef typename Acc<T>::type A_t;
  const int b = blockIdx.y;
  const GemvWork<T, MT> W = work[b];
  if (W.nchunk == 1) return;
  const GemvProb<T, MT>& P = W.p;
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
  // In-place Gauss-Jordan with partial (row) pivoting on a copy of A in Ainv;
  // the row interchanges are undone as column interchanges at the end.
  const InvProb P = probs[blockIdx.x];
  const int n = P.n, tid = threadIdx.x, nt = blockDim.x;
  double* M = P.Ainv;
  const int ld = P.ldinv;
  __shared__ double sval[32];
  __shared__ int sidx[32];
  __shared__ int s_flag;
  extern __shared__ double colc[];  // multipliers of the pivot column (n)
  int* ipiv = reinterpret_cast<int*>(P.W);  // n pivot rows (work buffer)
  if (tid == 0) s_flag = 0;
  for (int c = tid; c < n; c += nt) ipiv[c] = c;
  double amax = 0.0;
  for (int j = tid >> 5; j < n; j += nt >> 5)
    for (int i = tid & 31; i < n; i += 32) {
      const double v = P.A[i + size_t(j) * P.lda];
      M[i + size_t(j) * ld] = v;
      amax = fmax(amax, fabs(v));
    }
  int dummy;
  amax = block_reduce_max_abs_arg(amax, 0, &dummy, sval, sidx);
  const double tiny = 1e-14 * amax;
  for (int c = 0; c < n; ++c) {
    double v = -1.0;
    int idx = 0x7fffffff;
    for (int r = c + tid; r < n; r += nt) {
      const double a = fabs(M[r + size_t(c) * ld]);
      if (a > v) { v = a; idx = r; }
    }
    int p;
    const double pv = block_reduce_max_abs_arg(v, idx, &p, sval, sidx);
    if (!(pv > tiny)) {
      if (tid == 0) s_flag = 1;
      if (pv == 0.0) { __syncthreads(); break; }
    }
    if (tid == 0) ipiv[c] = p;
    if (p != c) {
      for (int j = tid; j < n; j += nt) {
        const double t = M[c + size_t(j) * ld];
        M[c + size_t(j) * ld] = M[p + size_t(j) * ld];
        M[p + size_t(j) * ld] = t;
      }
      __syncthreads();
    }
    const double invp = 1.0 / M[c + size_t(c) * ld];
    for (int r = tid; r < n; r += nt) colc[r] = (r == c) ? 0.0 : M[r + size_t(c) * ld];
    __syncthreads();
    for (int j = tid; j < n; j += nt) M[c + size_t(j) * ld] = (j == c) ? invp : M[c + size_t(j) * ld] * invp;
    __syncthreads();
    {
      // warps over columns, lanes over rows (coalesced, no index division)
      const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
      for (int j = warp; j < n; j += nw) {
        double* mj = M + size_t(j) * ld;
        if (j == c) {
          for (int r = lane; r < n; r += 32) if (r != c) mj[r] = -colc[r] * invp;
        } else {
          const double pj = mj[c];
          if (pj != 0.0) {
            // 8 rows per lane in flight: loads first, then the updates
            for (int r0 = 0; r0 < n; r0 += 256) {
              double v[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int r = r0 + lane + 32 * u;
                v[u] = (r < n) ? mj[r] : 0.0;
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int r = r0 + lane + 32 * u;
                if (r < n && r != c) mj[r] = v[u] - colc[r] * pj;
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int c = n - 1; c >= 0; --c) {
    const int p = ipiv[c];
    if (p != c)
      for (int r = tid; r < n; r += nt) {
        const double t = M[r + size_t(c) * ld];
        M[r + size_t(c) * ld] = M[r + size_t(p) * ld];
        M[r + size_t(p) * ld] = t;
      }
    __syncthreads();
  }
  if (tid == 0 && P.flag && s_flag) atomicOr(P.flag, 1);  // flags are only ever raised
}

// Cluster Gauss-Jordan (partial row pivoting): CTA r of a CS-CTA cluster
// owns columns [r cw, (r+1) cw), in shared memory (SM) or in place in Ainv.
// Per pivot column c: the owner finds the pivot row and publishes it;
// cluster barrier; every CTA swaps the two rows in its columns; the owner
// publishes the multiplier column and 1/pivot; cluster barrier; every CTA
// copies them through distributed shared memory and eliminates its columns.
// The row interchanges become a column permutation applied on write-back
// (through the work buffer W).
template <bool SM>
__global__ void __launch_bounds__(256) k_inverse_cluster(const InvProb* probs, int base, int CS) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = int(cluster.block_rank());
  const InvProb P = probs[base + blockIdx.x / CS];
  const int n = P.n, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int cw = (n + CS - 1) / CS;
  const int c0 = crank * cw, c1 = min(n, c0 + cw), ncl = max(0, c1 - c0);
  extern __shared__ double smem[];
  double* colc = smem;                       // 2 x n: published pivot column (owner), by step parity
  double* mine = colc + 2 * n;               // n: local copy of the multipliers
  int* ipiv = reinterpret_cast<int*>(mine + n);  // n
  double* Ml = reinterpret_cast<double*>(ipiv + ((n + 1) & ~1));  // n x cw (SM)
  double* M;
  int ld;
  if (SM) { M = Ml; ld = n; } else { M = P.Ainv + size_t(c0) * P.ldinv; ld = P.ldinv; }
  __shared__ double sval[32];
  __shared__ int sidx[32];
  __shared__ double pub_val, pub_pv[2];
  __shared__ int pub_p[2], g_p, s_flag;
  if (tid == 0) s_flag = 0;
  // load my columns, max |A| over my columns
  double amax = 0.0;
  for (int j = warp; j < ncl; j += nw)
    for (int i = lane; i < n; i += 32) {
      const double v = P.A[i + size_t(c0 + j) * P.lda];
      M[i + size_t(j) * ld] = v;
      amax = fmax(amax, fabs(v));
    }
  int dummy;
  amax = block_reduce_max_abs_arg(amax, 0, &dummy, sval, sidx);
  if (tid == 0) pub_val = amax;
  cluster.sync();
  if (tid == 0) {
    double a = 0.0;
    for (int r = 0; r < CS; ++r) a = fmax(a, *cluster.map_shared_rank(&pub_val, r));
    sval[31] = a;
  }
  __syncthreads();
  const double tiny = 1e-14 * sval[31];
  cluster.sync();  // pub_val is reused below
  // One cluster barrier per column: the owner publishes the column as it
  // is (before the row interchange) with its pivot row, double-buffered by
  // step parity; every CTA applies the interchange while copying it.
  for (int c = 0; c < n; ++c) {
    const int owner = c / cw, par = c & 1;
    if (crank == owner) {
      const int jl = c - c0;
      const double* mc = M + size_t(jl) * ld;
      double v = -1.0;
      int idx = 0x7fffffff;
      for (int r = c + tid; r < n; r += nt) {
        const double a = fabs(mc[r]);
        if (a > v) { v = a; idx = r; }
      }
      int p;
      const double pv = block_reduce_max_abs_arg(v, idx, &p, sval, sidx);
      double* pub = colc + size_t(par) * n;
      for (int r = tid; r < n; r += nt) pub[r] = mc[r];
      if (tid == 0) { pub_p[par] = p; pub_pv[par] = pv; }
    }
    cluster.sync();
    const int p = *cluster.map_shared_rank(&pub_p[par], owner);
    if (tid == 0) {
      if (!(*cluster.map_shared_rank(&pub_pv[par], owner) > tiny)) s_flag = 1;
      ipiv[c] = p;
    }
    const double* rc = cluster.map_shared_rank(colc + size_t(par) * n, owner);
    const double invp = 1.0 / rc[p];
    for (int r = tid; r < n; r += nt) mine[r] = (r == c) ? 0.0 : rc[r == p ? c : r];
    if (p != c)
      for (int j = tid; j < ncl; j += nt) {
        double* mj = M + size_t(j) * ld;
        const double t = mj[c];
        mj[c] = mj[p];
        mj[p] = t;
      }
    __syncthreads();
    for (int j = warp; j < ncl; j += nw) {
      double* mj = M + size_t(j) * ld;
      if (c0 + j == c) {
        for (int r = lane; r < n; r += 32) mj[r] = (r == c) ? invp : -mine[r] * invp;
      } else {
        const double pj = mj[c] * invp;
        if (pj != 0.0) {
          for (int r0 = 0; r0 < n; r0 += 256) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int r = r0 + lane + 32 * u;
              v[u] = (r < n) ? mj[r] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int r = r0 + lane + 32 * u;
              if (r < n) mj[r] = (r == c) ? pj : v[u] - mine[r] * pj;
            }
          }
        }
        __syncwarp();
        if (lane == 0 && pj == 0.0) mj[c] = 0.0;
      }
    }
    __syncthreads();
  }
  // column permutation from the row interchanges (last first); the barrier
  // keeps colc alive until every CTA has copied the last multipliers
  cluster.sync();
  int* perm = ipiv;
  if (tid == 0) {
    // sigma[j]: original column that ends up at position j
    // computed in place over a temporary in colc's memory (as ints)
    int* sigma = reinterpret_cast<int*>(colc);
    for (int j = 0; j < n; ++j) sigma[j] = j;
    for (int c = n - 1; c >= 0; --c) {
      const int q = perm[c];
      if (q != c) { const int t = sigma[c]; sigma[c] = sigma[q]; sigma[q] = t; }
    }
  }
  // write my columns to the work buffer (W, ld n), then gather by sigma
  for (int j = warp; j < ncl; j += nw)
    for (int i = lane; i < n; i += 32) P.W[i + size_t(c0 + j) * n] = M[i + size_t(j) * ld];
  __threadfence();
  cluster.sync();
  {
    const int* sigma = reinterpret_cast<const int*>(colc);
    for (int j = warp; j < ncl; j += nw) {
      const int src = sigma[c0 + j];
      for (int i = lane; i < n; i += 32) P.Ainv[i + size_t(c0 + j) * P.ldinv] = P.W[i + size_t(src) * n];
    }
  }
  if (tid == 0 && s_flag && P.flag) atomicOr(P.flag, 1);
  cluster.sync();
}

// ------------------------------------------------------------------ ID
// Column-pivoted Householder QR of W (nr x nc) with early stop, then
// T = R11^{-1} R12.  SM = true: W is staged in shared memory (small
// problems); else W stays in global memory and the current Householder
// vector is cached in shared memory.
template <bool SM>
__global__ void __launch_bounds__(512) k_cpqr_id(const IdProb* probs, int nprob_base, double* flops_out) {
  const IdProb P = probs[nprob_base + blockIdx.x];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int nr = P.nr, nc = P.nc;
  extern __shared__ double smem[];
  double* W;
  int ld;
  double* vcache;
  if (SM) {
    W = smem;
    ld = nr;
    vcache = nullptr;
    for (long long e = tid; e < (long long)nr * nc; e += nt) {
      const int i = int(e % nr), j = int(e / nr);
      W[e] = P.W[i + size_t(j) * P.ldw];
    }
  } else {
    W = P.W;
    ld = P.ldw;
    vcache = smem;
  }
  double* nrm = P.norms;
  double* nrm0 = P.norms + nc;
  int* piv = P.piv;
  __shared__ double sval[32];
  __shared__ int sidx[32];
  __shared__ double s_tau, s_scale;
  if (nr <= 0 || nc <= 0) {
    if (tid == 0) { *P.rank = 0; if (nc > 0) { P.norms[2 * nc] = 0.0; P.norms[2 * nc + 3] = 0.0; } }
    return;
  }
  for (int j = tid; j < nc; j += nt) piv[j] = j;
  __syncthreads();
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
    double* col = W + size_t(s) * ld;
    double part = 0.0;
    for (int i = s + 1 + tid; i < nr; i += nt) part += col[i] * col[i];
    const double xn2 = block_reduce_sum(part, sval);
    const double alpha = col[s];
    if (tid == 0) {
      if (xn2 == 0.0) {
        s_tau = 0.0;
        s_scale = 0.0;
      } else {
        double beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
        s_tau = (beta - alpha) / beta;
        s_scale = 1.0 / (alpha - beta);
        col[s] = beta;
      }
    }
    __syncthreads();
    const double tau = s_tau;
    const double* vv = col;
    if (tau != 0.0) {
      const double sc = s_scale;
      for (int i = s + 1 + tid; i < nr; i += nt) {
        const double x = col[i] * sc;
        col[i] = x;
        if (!SM) vcache[i] = x;
      }
      if (!SM) vv = vcache;
    }
    __syncthreads();
    for (int j = s + 1 + warp; j < nc; j += nw) {
      double* cj = W + size_t(j) * ld;
      if (tau != 0.0) {
        double d = 0.0;
        for (int i = s + 1 + lane; i < nr; i += 32) d += vv[i] * cj[i];
        for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
        d = __shfl_sync(0xffffffffu, d, 0);
        d = tau * (d + cj[s]);
        for (int i = s + 1 + lane; i < nr; i += 32) cj[i] -= d * vv[i];
        __syncwarp();
        if (lane == 0) cj[s] -= d;
        __syncwarp();
      }
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
  // T = R11^{-1} R12 over the first keff pivots, in place in W[0:keff, k:nc]
  for (int j = k + tid; j < nc; j += nt) {
    double* cj = W + size_t(j) * ld;
    for (int i = keff - 1; i >= 0; --i) {
      double acc = cj[i];
      for (int l = i + 1; l < keff; ++l) acc -= W[i + size_t(l) * ld] * cj[l];
      cj[i] = acc / W[i + size_t(i) * ld];
    }
  }
  __syncthreads();
  if (tid == 0) {
    *P.rank = k; P.norms[2 * nc] = double(keff); P.norms[2 * nc + 3] = 0.0;
    if (flops_out) {
      double f = 0.0;
      for (int q = 0; q < s; ++q) f += 4.0 * double(nr - q) * double(nc - q - 1);
      atomicAdd(flops_out, f);
    }
  }
  if (SM) {
    // the finished factorisation (R and T) goes back for k_id_interp
    for (long long e = tid; e < (long long)nr * nc; e += nt) {
      const int i = int(e % nr), j = int(e / nr);
      if (i < keff) P.W[i + size_t(j) * P.ldw] = W[e];
    }
  }
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

// Threads per column in the column updates of a CTA holding cw columns
// (a power of two <= 32, so that the CTA's threads cover its columns), and
// the shared-memory column stride for it: with G < 16 threads on
// consecutive rows of a column, a stride of G modulo 16 doubles puts the
// columns of one warp in distinct banks.
__host__ __device__ inline int cpqr_threads_per_col(int cw, int nt) {
  int G = 32;
  while (G > 1 && (nt / G) < cw) G >>= 1;
  return G;
}
__host__ __device__ inline int cpqr_ld(int nr, int G) {
  return G >= 16 ? nr : nr + ((G - nr % 16) + 16) % 16;
}
// Threads of a cluster-QR CTA.
constexpr int kCpqrThreads = 256;
// Shared memory of a cluster-QR CTA (bytes): its columns, two published
// columns, the Householder vector and two norm arrays.
__host__ __device__ inline size_t cpqr_cluster_smem(int nr, int cw, int nt) {
  return (size_t(cpqr_ld(nr, cpqr_threads_per_col(cw, nt))) * cw + 3 * size_t(nr) + 2 * size_t(cw)) * sizeof(double);
}

// One pivot step's update of a CTA's candidate columns (shared memory, nr
// rows each) by the Householder reflector I - tau v v^T (v(s) = 1, v(i) =
// vloc(i) below): G threads (a power of two <= 32, within one warp) per
// column compute the dot product and the update, then the column's squared
// norm is downdated by the square of the entry leaving it and recomputed
// exactly when cancellation makes the downdate unreliable (remaining square
// <= sqrt(eps) x the square at the last exact computation: LAPACK xLAQP2's
// test, stated on squares, which needs no division or square root).  Done
// columns carry a negative value.
__device__ __forceinline__ void cpqr_update_columns(double* Wl, int ld, int nr, int ncl, int ncl_pad, int G, int s,
                                                    double tau, const double* vloc, double* nrm, double* nrm0,
                                                    double tol3z, double& lv, int& li, int c0) {
  const int tid = threadIdx.x, nt = blockDim.x, gl = tid & (G - 1);
  lv = -1.0;
  li = 0x7fffffff;
  for (int j = tid / G; j < ncl_pad; j += nt / G) {
    const bool live = j < ncl && nrm[j] >= 0.0;
    double* cj = Wl + size_t(live ? j : 0) * ld;
    double dd = 0.0;
    if (live && tau != 0.0)
      for (int i = s + 1 + gl; i < nr; i += G) dd += vloc[i] * cj[i];
    for (int off = G / 2; off > 0; off >>= 1) dd += __shfl_down_sync(0xffffffffu, dd, off, G);
    dd = __shfl_sync(0xffffffffu, dd, 0, G);
    int recompute = 0;
    if (live) {
      if (tau != 0.0) {
        dd = tau * (dd + cj[s]);
        for (int i = s + 1 + gl; i < nr; i += G) cj[i] -= dd * vloc[i];
      }
      const double rs = (tau != 0.0) ? cj[s] - dd : cj[s];
      const double nj2 = nrm[j];
      if (nj2 != 0.0) {
        const double t2 = fmax(0.0, fma(-rs, rs, nj2));
        if (t2 <= tol3z * nrm0[j]) recompute = 1;
        else if (gl == 0) nrm[j] = t2;
      }
    }
    // recompute decisions differ between groups: every lane joins the
    // shuffles, lanes of groups without a recompute add zeros
    double q = 0.0;
    if (live && recompute)
      for (int i = s + 1 + gl; i < nr; i += G) q += cj[i] * cj[i];
    for (int off = G / 2; off > 0; off >>= 1) q += __shfl_down_sync(0xffffffffu, q, off, G);
    if (live && gl == 0) {
      if (tau != 0.0) cj[s] -= dd;
      if (recompute) { nrm[j] = q; nrm0[j] = q; }
      // this thread's next-pivot candidate (its columns in increasing order)
      const double nj = nrm[j];
      if (nj > lv) { lv = nj; li = c0 + j; }
    }
  }
}

// Cluster variant (thread-block cluster of CS CTAs per problem): CTA r of
// the cluster keeps candidate columns [r cw, (r+1) cw) of W in its shared
// memory, column stride cpqr_ld(nr, G) (padded so that the G threads of a
// column and the columns of a warp fall in distinct banks).  One cluster
// barrier per pivot step: every CTA publishes its local column-norm maximum
// together with a copy of that column (two buffers, by step parity); after
// the barrier warp 0 of every CTA reads all published maxima, so that every
// CTA takes the same decisions, copies the winning column through
// distributed shared memory and forms the Householder vector from it (the
// same arithmetic in every CTA); then every CTA updates its own columns,
// downdating their norms and finding its next local maximum in the same
// pass.  Columns are not swapped: column q keeps its data, piv[] records the
// pivot order, and the factorisation is written back to global memory in
// this "no-swap" layout (R(l, i) = W[l, piv[i]]; T for a non-pivot candidate
// q in column q).
//
// Paired mode (paired = 1): a cluster of 2 CS CTAs factors problems 2c and
// 2c+1 side by side (CTAs [0, CS) and [CS, 2 CS)) with a joint stopping
// rule: both continue while either has not met its tolerance, so both end
// with the larger of the two ranks (the common rank of a node's row and
// column IDs) in one pass.  A problem that runs out of candidates or of
// nonzero columns stops on its own while its partner continues.
__global__ void __launch_bounds__(kCpqrThreads) k_cpqr_cluster(const IdProb* probs, int base, int CS, int paired,
                                                      double* flops_out) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = int(cluster.block_rank());
  const int np = paired ? 2 : 1;
  const int half = crank / CS, lr = crank % CS;
  const int pidx = base + (blockIdx.x / (CS * np)) * np + half;
  const IdProb P = probs[pidx];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nr = P.nr, nc = P.nc;
  const int cw = (nc + CS - 1) / CS;
  const int c0 = min(nc, lr * cw), c1 = min(nc, c0 + cw), ncl = max(0, c1 - c0);
  const int G = cpqr_threads_per_col(cw, nt);
  const int ld = cpqr_ld(nr, G);
  extern __shared__ double smem[];
  double* Wl = smem;                   // ld x cw
  double* pubc = Wl + size_t(ld) * cw;  // 2 x nr: published column, by step parity
  double* vloc = pubc + 2 * size_t(nr);  // Householder vector of the current step
  double* nrm = vloc + nr;              // cw
  double* nrm0 = nrm + cw;              // cw
  __shared__ double pubv[2], g_val, g_val_o, g_tau, g_beta;
  __shared__ int pubi[2], g_idx;
  __shared__ double sval[32];
  __shared__ int sidx[32];
  for (int e = tid; e < nr * ncl; e += nt) {
    const int i = e % nr, j = e / nr;
    Wl[i + size_t(j) * ld] = P.W[i + size_t(c0 + j) * P.ldw];
  }
  __syncthreads();
  for (int j = warp; j < ncl; j += nt >> 5) {
    double q = 0.0;
    for (int i = lane; i < nr; i += 32) { const double v = Wl[i + size_t(j) * ld]; q += v * v; }
    for (int off = 16; off > 0; off >>= 1) q += __shfl_down_sync(0xffffffffu, q, off);
    if (lane == 0) { nrm[j] = q; nrm0[j] = q; }
  }
  __syncthreads();
  const int maxsteps = (nr <= 0 || nc <= 0) ? 0 : min(min(nr, nc), P.max_rank);
  int maxsteps_o = 0, minrank_o = 0;
  double tabs_o = 0.0, trel_o = 0.0;
  if (paired) {
    const IdProb& Q = probs[pidx + (half == 0 ? 1 : -1)];
    maxsteps_o = (Q.nr <= 0 || Q.nc <= 0) ? 0 : min(min(Q.nr, Q.nc), Q.max_rank);
    minrank_o = Q.min_rank;
    tabs_o = Q.tol_abs;
    trel_o = Q.tol_rel;
  }
  const double tol3z = sqrt(2.220446049250313e-16);
  const int ncl_pad = (ncl + (nt / G) - 1) / (nt / G) * (nt / G);
  // the local maximum of the initial norms (smallest global index on ties)
  double lv = -1.0;
  int li = 0x7fffffff;
  for (int j = tid; j < ncl; j += nt) if (nrm[j] > lv) { lv = nrm[j]; li = c0 + j; }
  double ref = 0.0, ref_o = 0.0;
  bool done = false, done_o = !paired;
  int s = 0;  // steps taken by this CTA's problem
  for (int it = 0;; ++it) {
    const int par = it & 1;
    // publish the local maximum and a copy of its column
    {
      int p;
      const double lm = block_reduce_max_abs_arg(done ? -1.0 : lv, done ? 0x7fffffff : li, &p, sval, sidx);
      double* pc = pubc + size_t(par) * nr;
      if (lm >= 0.0 && p >= c0 && p < c1)
        for (int i = tid; i < nr; i += nt) pc[i] = Wl[i + size_t(p - c0) * ld];
      if (tid == 0) { pubv[par] = lm; pubi[par] = p; }
    }
    cluster.sync();
    if (warp == 0) {
      // lane r reads CTA r's slot; arg-max over this problem's CTAs
      // (smallest index on ties) and the partner's maximum
      double bv = -1.0, ov_o = -1.0;
      int bi = 0x7fffffff;
      if (lane < CS * np) {
        const double x = *cluster.map_shared_rank(&pubv[par], lane);
        const int xi = *cluster.map_shared_rank(&pubi[par], lane);
        if (lane / CS == half) { bv = x; bi = xi; }
        else ov_o = x;
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        ov_o = fmax(ov_o, __shfl_down_sync(0xffffffffu, ov_o, off));
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      bv = __shfl_sync(0xffffffffu, bv, 0);
      bi = __shfl_sync(0xffffffffu, bi, 0);
      ov_o = __shfl_sync(0xffffffffu, ov_o, 0);
      // the stopping rule (the same in every CTA), then the Householder
      // vector of the winning column, formed by this warp
      if (it == 0) { ref = sqrt(fmax(bv, 0.0)); ref_o = sqrt(fmax(ov_o, 0.0)); }
      const double thr = fmax(P.tol_abs, P.tol_rel * ref), thr_o = fmax(tabs_o, trel_o * ref_o);
      const bool hard = done || it >= maxsteps || bv <= 0.0;
      const bool soft = hard || (it >= P.min_rank && bv <= thr * thr);
      const bool hard_o = done_o || it >= maxsteps_o || ov_o <= 0.0;
      const bool soft_o = hard_o || (it >= minrank_o && ov_o <= thr_o * thr_o);
      int stop = (soft && soft_o) ? 1 : 0;
      if (!stop && !hard) {
        const int owner = half * CS + bi / cw;
        const double* rc = cluster.map_shared_rank(pubc + size_t(par) * nr, owner);
        double xn2 = 0.0;
        for (int i = s + 1 + lane; i < nr; i += 32) { const double x = rc[i]; vloc[i] = x; xn2 += x * x; }
        for (int off = 16; off > 0; off >>= 1) xn2 += __shfl_down_sync(0xffffffffu, xn2, off);
        xn2 = __shfl_sync(0xffffffffu, xn2, 0);
        const double alpha = rc[s];
        double tau = 0.0, beta = alpha;
        if (xn2 != 0.0) {
          beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
          tau = (beta - alpha) / beta;
          const double sc = 1.0 / (alpha - beta);
          __syncwarp();
          for (int i = s + 1 + lane; i < nr; i += 32) vloc[i] *= sc;
        }
        if (lane == 0) { g_tau = tau; g_beta = beta; }
        if (bi >= c0 && bi < c1) {
          // the pivot column becomes R's column s over the reflector, and
          // leaves the candidates
          double* col = Wl + size_t(bi - c0) * ld;
          for (int i = s + 1 + lane; i < nr; i += 32) col[i] = vloc[i];
          if (lane == 0) {
            col[s] = beta;
            nrm[bi - c0] = -1.0;
          }
        }
        if (lane == 0 && lr == 0) P.piv[s] = bi;
      }
      if (lane == 0) { g_val = bv; g_val_o = ov_o; g_idx = stop ? -1 : bi; }
    }
    __syncthreads();
    if (g_idx < 0) break;
    const double vmax = g_val, vmax_o = g_val_o;
    const int pg = g_idx;
    if (it == 0) { ref = sqrt(fmax(vmax, 0.0)); ref_o = sqrt(fmax(vmax_o, 0.0)); }
    const bool hard = done || it >= maxsteps || vmax <= 0.0;
    const bool hard_o = done_o || it >= maxsteps_o || vmax_o <= 0.0;
    done = hard;
    done_o = hard_o;
    (void)pg;
    if (!done) {
      // the update finds each thread's next candidate; the next step's
      // block reduction (its barriers) orders it before the publication
      cpqr_update_columns(Wl, ld, nr, ncl, ncl_pad, G, s, g_tau, vloc, nrm, nrm0, tol3z, lv, li, c0);
      ++s;
    }
  }
  __syncthreads();
  for (int e = tid; e < nr * ncl; e += nt) {
    const int i = e % nr, j = e / nr;
    P.W[i + size_t(c0 + j) * P.ldw] = Wl[i + size_t(j) * ld];
  }
  // done flags for the remaining-pivot bookkeeping: mark in global norms
  for (int j = tid; j < ncl; j += nt) P.norms[nc + c0 + j] = (nrm[j] < 0.0) ? -1.0 : 1.0;
  if (lr == 0 && tid == 0) {
    P.norms[2 * nc + 1] = double(s); P.norms[2 * nc + 2] = ref; P.norms[2 * nc + 3] = 1.0;
    if (flops_out) {
      // Householder QR with column pivoting: dot + update = 4 flops per
      // trailing entry per step
      double f = 0.0;
      for (int q = 0; q < s; ++q) f += 4.0 * double(nr - q) * double(nc - q - 1);
      atomicAdd(flops_out, f);
    }
  }
  cluster.sync();  // keep shared memory alive until remote readers are done
}

// Grid-wide variant for a few problems (one to a few dozen, hundreds to
// thousands of candidates each): one cooperative grid, problem p owning the
// CTAs [b0_p, b0_p + G_p); CTA b keeps candidate columns [r cw_p,
// (r+1) cw_p) of its problem (r = b - b0_p) in shared memory.  One grid
// barrier per pivot step: every CTA publishes its local norm maximum
// together with that column (double-buffered by step parity); after the
// barrier every CTA reads all published maxima, so every CTA takes the same
// decisions for every problem, forms its problem's Householder vector from
// the published pivot column and updates its own columns.  Paired mode:
// problems 2i and 2i+1 stop jointly, as in the cluster variant.  Same
// no-swap layout and outputs.  pub holds 4 G + 2 G nr_max doubles.
constexpr int kGridIdMaxProbs = 64;
constexpr int kGridIdMaxCtas = 256;
__global__ void __launch_bounds__(256) k_cpqr_grid(const IdProb* probs, int base, int np, const int* parts,
                                                   int paired, int nr_max, double* pub, double* flops_out) {
  cg::grid_group grid = cg::this_grid();
  const int G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  __shared__ int s_b0[kGridIdMaxProbs], s_G[kGridIdMaxProbs], s_s[kGridIdMaxProbs], s_own[kGridIdMaxProbs];
  __shared__ int s_idx[kGridIdMaxProbs], s_act[kGridIdMaxProbs], s_soft[kGridIdMaxProbs], s_hard[kGridIdMaxProbs];
  __shared__ int s_mx[kGridIdMaxProbs], s_minr[kGridIdMaxProbs];
  __shared__ double s_val[kGridIdMaxProbs], s_ref[kGridIdMaxProbs], s_tabs[kGridIdMaxProbs], s_trel[kGridIdMaxProbs];
  __shared__ double slot_v[kGridIdMaxCtas];
  __shared__ int slot_i[kGridIdMaxCtas];
  __shared__ double sval[32];
  __shared__ int sidx[32];
  for (int q = tid; q < np; q += nt) {
    const IdProb& Q = probs[base + q];
    s_b0[q] = parts[2 * q];
    s_G[q] = parts[2 * q + 1];
    s_s[q] = 0;
    s_act[q] = 1;
    s_ref[q] = 0.0;
    s_mx[q] = (Q.nr <= 0 || Q.nc <= 0) ? 0 : min(min(Q.nr, Q.nc), Q.max_rank);
    s_minr[q] = Q.min_rank;
    s_tabs[q] = Q.tol_abs;
    s_trel[q] = Q.tol_rel;
  }
  __syncthreads();
  int me = 0;
  while (me + 1 < np && b >= s_b0[me + 1]) ++me;
  const IdProb P = probs[base + me];
  const int Gp = s_G[me], lr = b - s_b0[me];
  const int nr = P.nr, nc = P.nc;
  const int cw = (nc + Gp - 1) / Gp;
  const int c0 = min(nc, lr * cw), c1 = min(nc, c0 + cw), ncl = max(0, c1 - c0);
  extern __shared__ double smem[];
  double* Wl = smem;                    // nr x cw
  double* vloc = Wl + size_t(nr) * cw;  // nr
  double* nrm = vloc + nr;              // cw
  double* nrm0 = nrm + cw;              // cw
  for (int e = tid; e < nr * ncl; e += nt) {
    const int i = e % nr, j = e / nr;
    Wl[i + size_t(j) * nr] = P.W[i + size_t(c0 + j) * P.ldw];
  }
  __syncthreads();
  for (int j = warp; j < ncl; j += nw) {
    double s = 0.0;
    for (int i = lane; i < nr; i += 32) { double v = Wl[i + size_t(j) * nr]; s += v * v; }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) { nrm[j] = s; nrm0[j] = s; }
  }
  __syncthreads();
  const double tol3z = sqrt(2.220446049250313e-16);
  int G2 = 32;
  while (G2 > 1 && (nt / G2) < ncl) G2 >>= 1;
  const int ncl_pad = (ncl + (nt / G2) - 1) / (nt / G2) * (nt / G2);
  for (int it = 0;; ++it) {
    const int par = it & 1;
    double* pv = pub + size_t(par) * G;
    double* pi = pub + 2 * size_t(G) + size_t(par) * G;
    double* pcol = pub + 4 * size_t(G) + (size_t(par) * G + b) * nr_max;
    const bool act = s_act[me] != 0;
    const int s = s_s[me];
    double v = -1.0;
    int id = 0x7fffffff;
    if (act)
      for (int j = tid; j < ncl; j += nt) if (nrm[j] > v) { v = nrm[j]; id = c0 + j; }
    int p;
    const double lm = block_reduce_max_abs_arg(v, id, &p, sval, sidx);
    if (lm >= 0.0) {
      const double* src = Wl + size_t(p - c0) * nr;
      for (int i = s + tid; i < nr; i += nt) pcol[i] = src[i];
    }
    if (tid == 0) { pv[b] = lm; pi[b] = double(lm >= 0.0 ? p : 0x7fffffff); }
    __threadfence();
    grid.sync();
    // every CTA's published maximum into shared memory (one pass), then
    // every problem's maximum (warp q % nw reduces problem q)
    for (int q = tid; q < G; q += nt) {
      slot_v[q] = __ldcg(pv + q);
      slot_i[q] = int(__ldcg(pi + q));
    }
    __syncthreads();
    for (int q = warp; q < np; q += nw) {
      double bv = -1.0;
      int bi = 0x7fffffff, bb = 0;
      for (int r = lane; r < s_G[q]; r += 32) {
        const int slot = s_b0[q] + r;
        const double ov = slot_v[slot];
        const int oi = slot_i[slot];
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; bb = slot; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        const int ob = __shfl_down_sync(0xffffffffu, bb, off);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; bb = ob; }
      }
      if (lane == 0) { s_val[q] = bv; s_idx[q] = bi; s_own[q] = bb; }
    }
    __syncthreads();
    // the same decisions in every CTA: soft = tolerance met (or no further
    // step possible), hard = no further step possible
    if (tid < np) {
      const int q = tid;
      // squared norms are published; s_ref is the first pivot norm itself
      if (it == 0) s_ref[q] = sqrt(fmax(s_val[q], 0.0));
      const double thr = fmax(s_tabs[q], s_trel[q] * s_ref[q]);
      const bool hard = !s_act[q] || s_s[q] >= s_mx[q] || s_val[q] <= 0.0;
      s_hard[q] = hard;
      s_soft[q] = hard || (s_s[q] >= s_minr[q] && s_val[q] <= thr * thr);
    }
    __syncthreads();
    int act_q = 0;
    if (tid < np) {
      const int q = tid, qp = ((q ^ 1) < np) ? (q ^ 1) : q;
      const bool stop = paired ? (s_soft[q] && s_soft[qp]) : s_soft[q];
      act_q = !(stop || s_hard[q]);
    }
    __syncthreads();
    if (tid < np) s_act[tid] = act_q;
    if (!__syncthreads_or(act_q)) break;
    if (s_act[me]) {
      const int pg = s_idx[me], owner = s_own[me];
      if (lr == 0 && tid == 0) P.piv[s] = pg;
      const double* col = pub + 4 * size_t(G) + (size_t(par) * G + owner) * nr_max;
      double part = 0.0;
      for (int i = s + 1 + tid; i < nr; i += nt) { const double x = __ldcg(col + i); part += x * x; }
      const double xn2 = block_reduce_sum(part, sval);
      const double alpha = __ldcg(col + s);
      double tau = 0.0, sc = 0.0, beta = alpha;
      if (xn2 != 0.0) {
        beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
        tau = (beta - alpha) / beta;
        sc = 1.0 / (alpha - beta);
      }
      for (int i = s + 1 + tid; i < nr; i += nt) vloc[i] = __ldcg(col + i) * sc;
      __syncthreads();
      if (b == owner) {
        const int jl = pg - c0;
        double* cp = Wl + size_t(jl) * nr;
        for (int i = s + 1 + tid; i < nr; i += nt) cp[i] = vloc[i];
        if (tid == 0) { cp[s] = beta; nrm[jl] = -1.0; }
        __syncthreads();
      }
      double lv_unused;
      int li_unused;
      cpqr_update_columns(Wl, nr, nr, ncl, ncl_pad, G2, s, tau, vloc, nrm, nrm0, tol3z, lv_unused, li_unused, 0);
    }
    __syncthreads();
    if (tid < np && s_act[tid]) s_s[tid] += 1;
    __syncthreads();
  }
  const int s = s_s[me];
  for (int e = tid; e < nr * ncl; e += nt) {
    const int i = e % nr, j = e / nr;
    P.W[i + size_t(c0 + j) * P.ldw] = Wl[i + size_t(j) * nr];
  }
  for (int j = tid; j < ncl; j += nt) P.norms[nc + c0 + j] = (nrm[j] < 0.0) ? -1.0 : 1.0;
  if (lr == 0 && tid == 0) {
    P.norms[2 * nc + 1] = double(s); P.norms[2 * nc + 2] = s_ref[me]; P.norms[2 * nc + 3] = 1.0;
    if (flops_out) {
      double f = 0.0;
      for (int q = 0; q < s; ++q) f += 4.0 * double(nr - q) * double(nc - q - 1);
      atomicAdd(flops_out, f);
    }
  }
}

// Completes a no-swap factorisation (one thread per problem): appends the
// non-pivot candidates to piv (increasing index), pads fixed-rank requests
// and counts the usable pivots.
__global__ void k_id_prep(const IdProb* probs, int base, int n) {
  // one warp per problem: ballot-compacted append of the non-pivot
  // candidates (increasing index) and a parallel search for the first
  // numerically zero pivot
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= n) return;
  const IdProb P = probs[base + b];
  const int nc = P.nc;
  const int s = int(P.norms[2 * nc + 1]);
  const double ref = P.norms[2 * nc + 2];
  const int k = max(s, min(P.min_rank, nc));
  int q = s;
  for (int j0 = 0; j0 < nc; j0 += 32) {
    const int j = j0 + lane;
    const bool keep = j < nc && P.norms[nc + j] >= 0.0;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) P.piv[q + __popc(m & ((1u << lane) - 1u))] = j;
    q += __popc(m);
  }
  int first = s;
  for (int i = lane; i < s; i += 32)
    if (!(fabs(P.W[i + size_t(P.piv[i]) * P.ldw]) > 1e-15 * ref)) { first = i; break; }
  for (int off = 16; off > 0; off >>= 1) first = min(first, __shfl_down_sync(0xffffffffu, first, off));
  if (lane == 0) {
    *P.rank = k;
    P.norms[2 * nc] = double(first);
  }
}

// T = R11^{-1} R12 for no-swap factorisations: blockIdx.y = problem,
// blockIdx.x = chunk of TS_COLS non-skeleton candidates.  Column-parallel
// back substitution: the chunk's right-hand sides sit in shared memory, and
// at step i (from keff-1 down) every thread scales its column's entry i by
// 1 / R(i, i) and updates its share of rows l < i.  R11 (pivot order) is
// staged in shared memory as a packed upper triangle when keff <= rmax, else
// read from global memory.
constexpr int TS_COLS = 16;
__global__ void __launch_bounds__(256) k_id_tsolve(const IdProb* probs, int base, int rmax) {
  const IdProb P = probs[base + blockIdx.y];
  const int nc = P.nc, k = *P.rank, keff = int(P.norms[2 * nc]);
  const int q0 = k + blockIdx.x * TS_COLS;
  if (q0 >= nc || keff == 0) return;
  const int ncols = min(TS_COLS, nc - q0);
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int c = tid % TS_COLS, rg = tid / TS_COLS, nrg = nt / TS_COLS;
  extern __shared__ double sm[];
  const bool inR = keff <= rmax;
  double* R = sm;                                                   // packed, column i at i(i+1)/2
  double* B = sm + (inR ? size_t(keff) * (keff + 1) / 2 : 0);       // keff x TS_COLS, B[l TS_COLS + c]
  double* dinv = B + size_t(keff) * TS_COLS;                        // keff
  if (inR)
    for (int i = warp; i < keff; i += nw) {
      const double* src = P.W + size_t(P.piv[i]) * P.ldw;
      double* dst = R + size_t(i) * (i + 1) / 2;
      for (int l = lane; l <= i; l += 32) dst[l] = src[l];
    }
  for (int i = tid; i < keff; i += nt) dinv[i] = 1.0 / P.W[i + size_t(P.piv[i]) * P.ldw];
  for (int e = tid; e < keff * TS_COLS; e += nt) {
    const int l = e % keff, cc = e / keff;
    B[size_t(l) * TS_COLS + cc] = cc < ncols ? P.W[l + size_t(P.piv[q0 + cc]) * P.ldw] : 0.0;
  }
  __syncthreads();
  double* out = P.W + size_t(P.piv[q0 + min(c, ncols - 1)]) * P.ldw;
  const bool act = c < ncols;
  for (int i = keff - 1; i >= 0; --i) {
    const double ti = B[size_t(i) * TS_COLS + c] * dinv[i];
    const double* Ri = inR ? R + size_t(i) * (i + 1) / 2 : P.W + size_t(P.piv[i]) * P.ldw;
    for (int l = rg; l < i; l += nrg) B[size_t(l) * TS_COLS + c] -= Ri[l] * ti;
    if (act && rg == i % nrg) out[i] = ti;
    __syncthreads();
  }
}

// Interpolation matrix from a finished factorisation (rank in *rank, number
// of usable pivots in norms[0]).
__global__ void k_id_interp(const IdProb* probs) {
  const IdProb P = probs[blockIdx.y];
  const int nc = P.nc, k = *P.rank, keff = int(P.norms[2 * nc]);
  const bool noswap = P.norms[2 * nc + 3] != 0.0;
  for (int c = blockIdx.x; c < k; c += gridDim.x)
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    double v;
    if (j < k) v = (j == c) ? 1.0 : 0.0;
    else v = (c < keff) ? P.W[c + size_t(noswap ? P.piv[j] : j) * P.ldw] : 0.0;
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

__global__ void k_axpby(const double* x, double* y, size_t n, double a, double b) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) y[i] = a * x[i] + b * y[i];
}

__global__ void k_fill_zero(double* p, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) p[i] = 0.0;
}
__global__ void k_d2f(const double* in, float* out, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) out[i] = float(in[i]);
}

int grid_for(size_t n) { return int(std::min<size_t>((n + 255) / 256, 152 * 16)); }

}  // namespace

// Raise the dynamic shared-memory limit of every kernel that uses more than
// 48 KB, once per process, to the largest size any launch asks
// for.  Done once (not per launch) because the limit is a per-function
// setting shared by all host threads.
static void init_smem_limits() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    const int lim = 210 * 1024;
    cudaError_t e[4];
    e[0] = cudaFuncSetAttribute(k_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    e[1] = cudaFuncSetAttribute(k_cpqr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    e[2] = cudaFuncSetAttribute(k_id_tsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    e[3] = cudaFuncSetAttribute(k_cpqr_id<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    for (cudaError_t x : e) if (x != cudaSuccess) err = x;
    cudaError_t g0 = cudaFuncSetAttribute(k_cpqr_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (g0 != cudaSuccess) err = g0;
    cudaError_t f0 = cudaFuncSetAttribute(k_inverse_cluster<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaError_t f1 = cudaFuncSetAttribute(k_inverse_cluster<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (f0 != cudaSuccess) err = f0;
    if (f1 != cudaSuccess) err = f1;
    // 16-CTA clusters are only used when asked for (RW_GJ_CS=16): a part that
    // refuses the attribute keeps working with portable sizes
    cudaFuncSetAttribute(k_inverse_cluster<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_inverse_cluster<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
  });
  if (err != cudaSuccess) throw Error(RW_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(err));
}

namespace { int sm_count(); }

void batched_gemm(const std::vector<GemmProb>& probs, cudaStream_t s) {
  std::vector<GemmWork> ws;
  std::vector<int> offs(1, 0);
  long long tiles_all = 0;
  for (const auto& p : probs) {
    if (p.m <= 0 || p.n <= 0) continue;
    GemmWork w;
    w.p = p;
    w.tilesM = ceil_div(p.m, GBM);
    w.tilesN = ceil_div(p.n, GBN);
    w.nsplit = 1;
    w.kchunk = std::max(p.k, 1);
    w.scratch_off = 0;
    ws.push_back(w);
    tiles_all += (long long)w.tilesM * w.tilesN;
  }
  if (ws.empty()) return;
  // Split long inner dimensions when the output tiles alone cannot fill the
  // GPU (three CTAs per SM: one CTA runs at the SM's FP64 rate, so a launch
  // with fewer CTAs than SMs leaves FP64 units idle); chunks of at least 64,
  // partial sums added in a fixed order.
  // The chunk count of each problem follows its share of the work (tiles x
  // inner dimension), so that the CTAs of one launch carry similar work.
  size_t scratch = 0;
  const long long target = 3LL * sm_count();
  double tile_k = 0.0;
  for (auto& w : ws) tile_k += double(w.tilesM) * w.tilesN * std::max(w.p.k, 1);
  const double per_cta = tile_k / double(target);
  for (auto& w : ws) {
    const long long tiles = (long long)w.tilesM * w.tilesN;
    if (tiles_all < target && w.p.k >= 128) {
      int ns = int(std::min<double>(std::ceil(double(w.p.k) / std::max(per_cta, 1.0)), double(w.p.k / 64)));
      ns = std::min(ns, 128);
      if (ns > 1) {
        w.kchunk = ((w.p.k + ns - 1) / ns + GBK - 1) / GBK * GBK;
        w.nsplit = (w.p.k + w.kchunk - 1) / w.kchunk;
        w.scratch_off = (long long)scratch;
        scratch += size_t(w.nsplit) * w.p.m * w.p.n;
      }
    }
    offs.push_back(offs.back() + int(tiles * w.nsplit));
  }
  TBuf<double> sc(scratch, s);
  auto dw = to_device_tmp(ws, s);
  auto doff = to_device_tmp(offs, s);
  double fl = 0.0, by = 0.0;
  for (auto& w : ws) {
    fl += 2.0 * w.p.m * w.p.n * double(w.p.k);
    by += 8.0 * (double(w.p.m) * w.p.k + double(w.p.k) * w.p.n + 2.0 * w.p.m * w.p.n);
  }
  ProfScope ps(KC_GEMM, s, fl, by);
  k_gemm<<<offs.back(), 256, 0, s>>>(dw.p, doff.p, int(ws.size()), sc.p);
  RW_CHECK_LAUNCH();
  if (scratch) {
    long long mx = 0;
    for (auto& w : ws) mx = std::max(mx, (long long)w.p.m * w.p.n);
    int mn = 0;
    for (auto& w : ws) mn = std::max(mn, w.p.n);
    k_gemm_reduce<<<dim3(std::min(mn, 1024), int(ws.size())), 256, 0, s>>>(dw.p, sc.p);
    (void)mx;
    RW_CHECK_LAUNCH();
  }
}

template <class T, class MT>
static void gemv_plan(const std::vector<GemvProb<T, MT>>& probs, int nrhs, std::vector<GemvWork<T, MT>>& work,
                      std::vector<int>& offs, size_t& scratch) {
  offs.assign(1, 0);
  scratch = 0;
  for (const auto& p : probs) {
    if (p.m <= 0) continue;
    GemvWork<T, MT> w;
    w.p = p;
    w.tilesM = ceil_div(p.m, VR);
    w.nchunk = std::max(1, ceil_div(std::max(p.n, 1), VCHUNK));
    w.scratch_off = (long long)scratch;
    if (w.nchunk > 1) scratch += size_t(w.nchunk) * nrhs * p.m;
    work.push_back(w);
    offs.push_back(offs.back() + w.tilesM * w.nchunk);
  }
}

template <class T, class MT>
size_t gemv_scratch_elems(const std::vector<GemvProb<T, MT>>& probs, int nrhs) {
  std::vector<GemvWork<T, MT>> w;
  std::vector<int> o;
  size_t sc;
  gemv_plan(probs, nrhs, w, o, sc);
  return sc;
}

template <class T, class MT>
void batched_gemv(const std::vector<GemvProb<T, MT>>& probs, int nrhs, T* scratch, cudaStream_t s) {
  require(nrhs >= 1 && nrhs <= 8, "batched_gemv: nrhs must be in 1..8");
  std::vector<GemvWork<T, MT>> work;
  std::vector<int> offs;
  size_t sc;
  gemv_plan(probs, nrhs, work, offs, sc);
  if (work.empty()) return;
  require(sc == 0 || scratch != nullptr, "batched_gemv: scratch buffer missing");
  auto dw = to_device_tmp(work, s);
  auto doff = to_device_tmp(offs, s);
  const int nprob = int(work.size());
  int maxm = 0;
  double fl = 0.0, by = 0.0;
  for (auto& w : work) {
    maxm = std::max(maxm, w.p.m);
    fl += 2.0 * w.p.m * double(w.p.n) * nrhs;
    by += double(sizeof(MT)) * double(w.p.m) * w.p.n + double(sizeof(T)) * double(nrhs) * (w.p.n + 2.0 * w.p.m);
  }
  ProfScope ps(KC_GEMV, s, fl, by);
  switch (nrhs) {
#define RW_GEMV_CASE(NR)                                                                   \
  case NR:                                                                                 \
    k_gemv<T, MT, NR><<<offs.back(), 256, 0, s>>>(dw.p, doff.p, nprob, scratch);           \
    if (sc) k_gemv_reduce<T, MT, NR><<<dim3(ceil_div(maxm, 256), nprob), 256, 0, s>>>(dw.p, nprob, scratch); \
    break;
    RW_GEMV_CASE(1) RW_GEMV_CASE(2) RW_GEMV_CASE(3) RW_GEMV_CASE(4)
    RW_GEMV_CASE(5) RW_GEMV_CASE(6) RW_GEMV_CASE(7) RW_GEMV_CASE(8)
#undef RW_GEMV_CASE
  }
  RW_CHECK_LAUNCH();
}

template <class T>
void gemv_into_sizes(const std::vector<GemvProb<T>>& probs, int nrhs, size_t* desc_bytes, size_t* scratch_elems) {
  std::vector<GemvWork<T>> work;
  std::vector<int> offs;
  size_t sc;
  gemv_plan(probs, nrhs, work, offs, sc);
  *desc_bytes = work.size() * sizeof(GemvWork<T>) + offs.size() * sizeof(int) + 16;
  *scratch_elems = sc;
}

template <class T>
void gemv_into(const std::vector<GemvProb<T>>& probs, int nrhs, void* desc, T* scratch, cudaStream_t s) {
  require(nrhs >= 1 && nrhs <= 8, "gemv_into: nrhs must be in 1..8");
  std::vector<GemvWork<T>> work;
  std::vector<int> offs;
  size_t sc;
  gemv_plan(probs, nrhs, work, offs, sc);
  if (work.empty()) return;
  require(sc == 0 || scratch != nullptr, "gemv_into: scratch buffer missing");
  auto* dw = static_cast<GemvWork<T>*>(desc);
  int* doff = reinterpret_cast<int*>(static_cast<char*>(desc) + ((work.size() * sizeof(GemvWork<T>) + 15) / 16) * 16);
  RW_CUDA(cudaMemcpyAsync(dw, work.data(), work.size() * sizeof(GemvWork<T>), cudaMemcpyHostToDevice, s));
  RW_CUDA(cudaMemcpyAsync(doff, offs.data(), offs.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  const int nprob = int(work.size());
  int maxm = 0;
  for (auto& w : work) maxm = std::max(maxm, w.p.m);
  switch (nrhs) {
#define RW_GEMV_INTO_CASE(NR)                                                                \
  case NR:                                                                                   \
    k_gemv<T, T, NR><<<offs.back(), 256, 0, s>>>(dw, doff, nprob, scratch);                  \
    if (sc) k_gemv_reduce<T, T, NR><<<dim3(ceil_div(maxm, 256), nprob), 256, 0, s>>>(dw, nprob, scratch); \
    break;
    RW_GEMV_INTO_CASE(1) RW_GEMV_INTO_CASE(2) RW_GEMV_INTO_CASE(3) RW_GEMV_INTO_CASE(4)
    RW_GEMV_INTO_CASE(5) RW_GEMV_INTO_CASE(6) RW_GEMV_INTO_CASE(7) RW_GEMV_INTO_CASE(8)
#undef RW_GEMV_INTO_CASE
  }
  RW_CHECK_LAUNCH();
}

template void gemv_into_sizes<double>(const std::vector<GemvProb<double>>&, int, size_t*, size_t*);
template void gemv_into<double>(const std::vector<GemvProb<double>>&, int, void*, double*, cudaStream_t);

template size_t gemv_scratch_elems<double>(const std::vector<GemvProb<double>>&, int);
template size_t gemv_scratch_elems<float>(const std::vector<GemvProb<float>>&, int);
template size_t gemv_scratch_elems<float, __nv_bfloat16>(const std::vector<GemvProb<float, __nv_bfloat16>>&, int);
template void batched_gemv<double>(const std::vector<GemvProb<double>>&, int, double*, cudaStream_t);
template void batched_gemv<float>(const std::vector<GemvProb<float>>&, int, float*, cudaStream_t);
template void batched_gemv<float, __nv_bfloat16>(const std::vector<GemvProb<float, __nv_bfloat16>>&, int, float*,
                                                 cudaStream_t);

template <>
void matvec<double, double>(const std::vector<GemvProb<double>>& probs, int nrhs, cudaStream_t s) {
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

void block_inverse(const double* A, double* Ainv, int n, int nb, int* flag, cudaStream_t s) {
  require(n >= 1 && nb >= 1, "block_inverse: bad size");
  nb = std::min(nb, n);
  double* M = Ainv;  // worked on in place
  RW_CUDA(cudaMemcpyAsync(M, A, sizeof(double) * size_t(n) * n, cudaMemcpyDeviceToDevice, s));
  TBuf<double> C(size_t(n) * nb, s), T(size_t(nb) * n, s), P(size_t(nb) * nb, s), Wk(size_t(nb) * nb, s);
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int b = std::min(nb, n - j0), j1 = j0 + b;
    // C = M[:, J]; P = M[J, J]^{-1}
    RW_CUDA(cudaMemcpyAsync(C.p, M + size_t(j0) * n, sizeof(double) * size_t(n) * b, cudaMemcpyDeviceToDevice, s));
    batched_inverse({InvProb{C.p + j0, P.p, Wk.p, b, n, b, flag}}, s);
    // T = P M[J, :], with T[:, J] = P; then M[J, :] = T
    batched_gemm({GemmProb{P.p, M + j0, T.p, b, n, b, b, n, b, 0, 0, 1.0, 0.0}}, s);
    RW_CUDA(cudaMemcpy2DAsync(T.p + size_t(j0) * b, sizeof(double) * b, P.p, sizeof(double) * b,
                              sizeof(double) * b, b, cudaMemcpyDeviceToDevice, s));
    RW_CUDA(cudaMemcpy2DAsync(M + j0, sizeof(double) * n, T.p, sizeof(double) * b, sizeof(double) * b, n,
                              cudaMemcpyDeviceToDevice, s));
    // other rows: M[I, J] = 0, then M[I, :] -= C[I, :] T (so M[I, J] = -C[I] P)
    if (j0 > 0)
      RW_CUDA(cudaMemset2DAsync(M + size_t(j0) * n, sizeof(double) * n, 0, sizeof(double) * j0, b, s));
    if (j1 < n)
      RW_CUDA(cudaMemset2DAsync(M + j1 + size_t(j0) * n, sizeof(double) * n, 0, sizeof(double) * (n - j1), b, s));
    std::vector<GemmProb> g;
    if (j0 > 0) g.push_back(GemmProb{C.p, T.p, M, j0, n, b, n, b, n, 0, 0, -1.0, 1.0});
    if (j1 < n) g.push_back(GemmProb{C.p + j1, T.p, M + j1, n - j1, n, b, n, b, n, 0, 0, -1.0, 1.0});
    batched_gemm(g, s);
  }
}

void batched_inverse(const std::vector<InvProb>& probs, cudaStream_t s) {
  // small matrices: one CTA each; larger: a cluster of up to 8 CTAs with the
  // columns in shared memory when they fit, else in place in global memory
  std::vector<InvProb> small, cl_sm[5], cl_gl[5];
  const int sizes[5] = {1, 2, 4, 8, 16};
  const size_t cap = 200 * 1024;
  for (const auto& p : probs) {
    if (p.n <= 0) continue;
    if (p.n < 48) { small.push_back(p); continue; }
    // eight CTAs per matrix (measured fastest from n = 48 up: the pivot
    // steps are latency bound, more SMs shorten each elimination);
    // RW_GJ_CS (tuning) fixes another size: 1, 2, 4, 8 or 16 (non-portable)
    static const int fixed_cs = [] {
      const char* e = std::getenv("RW_GJ_CS");
      const int v = e ? std::atoi(e) : 0;
      return v == 1 ? 0 : v == 2 ? 1 : v == 4 ? 2 : v == 8 ? 3 : v == 16 ? 4 : 3;
    }();
    const int q = fixed_cs;
    const int CS = sizes[q];
    const int cw = (p.n + CS - 1) / CS;
    const size_t need = (3 * size_t(p.n) + size_t(p.n) * cw) * sizeof(double) + size_t(p.n + 2) * sizeof(int);
    if (need <= cap) cl_sm[q].push_back(p); else cl_gl[q].push_back(p);
  }
  init_smem_limits();
  if (!small.empty()) {
    auto dp = to_device_tmp(small, s);
    int maxn = 0;
    double fl = 0.0;
    for (auto& p : small) { maxn = std::max(maxn, p.n); fl += 2.0 * double(p.n) * p.n * p.n; }
    ProfScope prof(KC_INVERSE, s, fl, 0.0);
    k_inverse<<<int(small.size()), 512, size_t(maxn) * sizeof(double), s>>>(dp.p);
    RW_CHECK_LAUNCH();
  }
  for (int sm = 0; sm < 2; ++sm)
    for (int q = 0; q < 5; ++q) {
      auto& g = sm ? cl_sm[q] : cl_gl[q];
      if (g.empty()) continue;
      const int CS = sizes[q];
      size_t smem = 0;
      double fl = 0.0;
      for (auto& p : g) {
        const int cw = (p.n + CS - 1) / CS;
        smem = std::max(smem, (3 * size_t(p.n) + (sm ? size_t(p.n) * cw : 0)) * sizeof(double) +
                                  size_t(p.n + 2) * sizeof(int));
        fl += 2.0 * double(p.n) * p.n * p.n;
      }
      auto dp = to_device_tmp(g, s);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(unsigned(g.size() * CS));
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = CS;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      ProfScope prof(KC_INVERSE, s, fl, 0.0);
      if (sm) RW_CUDA(cudaLaunchKernelEx(&cfg, k_inverse_cluster<true>, (const InvProb*)dp.p, 0, CS));
      else RW_CUDA(cudaLaunchKernelEx(&cfg, k_inverse_cluster<false>, (const InvProb*)dp.p, 0, CS));
      RW_CHECK_LAUNCH();
    }
}

namespace {
int sm_count() {
  static std::once_flag once;
  static int n = 0;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 0;
  });
  if (n <= 0) throw Error(RW_ERR_CUDA, "cannot query the number of SMs");
  return n;
}

// Finishes a no-swap factorisation of ng problems at probs[base..): pivot
// bookkeeping and the interpolation coefficients T.
void id_finish(const IdProb* dprobs, int base, const std::vector<IdProb>& ps, cudaStream_t s) {
  int maxk = 0, maxnc = 0;
  for (auto& p : ps) {
    maxk = std::max(maxk, std::min(std::min(p.nr, p.nc), p.max_rank));
    maxnc = std::max(maxnc, p.nc);
  }
  const int ng = int(ps.size());
  ProfScope pf(KC_OTHER, s);
  k_id_prep<<<ceil_div(32LL * ng, 128), 128, 0, s>>>(dprobs, base, ng);
  RW_CHECK_LAUNCH();
  // R11 in shared memory (packed) when the rank found is at most rmax
  const int kk = std::max(maxk, 1);
  const int rmax = std::min(kk, 200);
  const size_t in_sm = size_t(rmax) * (rmax + 1) / 2 + size_t(rmax) * (TS_COLS + 1);
  const size_t out_sm = size_t(kk) * (TS_COLS + 1);
  const size_t tsm = std::max(in_sm, out_sm) * sizeof(double);
  k_id_tsolve<<<dim3(ceil_div(maxnc, TS_COLS), ng), 256, tsm, s>>>(dprobs, base, rmax);
  RW_CHECK_LAUNCH();
}

// Grid-wide plan for a few problems: CTA ranges (b0, G_p) per problem, the
// CTAs first covering each problem's shared-memory need and the rest shared
// out in proportion to the problems' sizes; false when the problems do not
// fit on the SMs within the shared-memory cap.
bool grid_id_plan(const std::vector<IdProb>& ps, size_t cap, std::vector<int>& parts, int* G, size_t* smem,
                  int* nr_max) {
  const int np = int(ps.size());
  if (np < 1 || np > kGridIdMaxProbs) return false;
  const int nsm = sm_count();
  std::vector<int> g(np);
  long long need = 0;
  double work = 0.0;
  for (int q = 0; q < np; ++q) {
    const IdProb& p = ps[q];
    if (p.nr <= 0 || p.nc <= 0 || std::min(p.nr, p.nc) > 1500) return false;  // T-solve staging bound
    const long long room = (long long)(cap / sizeof(double)) - p.nr;
    const long long cwmax = room / (p.nr + 2);
    if (cwmax < 1) return false;
    g[q] = ceil_div(p.nc, cwmax);
    need += g[q];
    work += double(p.nr) * p.nc;
  }
  if (need > nsm || nsm > kGridIdMaxCtas) return false;
  // CTAs beyond the shared-memory need are shared out up to the SM count, or
  // up to RW_ID_GRID_CTAS (tuning: leaves SMs to the other streams)
  static const int cap_ctas = [] {
    const char* e = std::getenv("RW_ID_GRID_CTAS");
    return e ? std::atoi(e) : 0;
  }();
  const long long budget = cap_ctas > 0 ? std::max<long long>(need, std::min(cap_ctas, nsm)) : nsm;
  const long long spare = budget - need;
  for (int q = 0; q < np; ++q) {
    const long long extra = (long long)(double(spare) * double(ps[q].nr) * ps[q].nc / work);
    g[q] = int(std::min<long long>(g[q] + extra, ps[q].nc));
  }
  parts.assign(2 * np, 0);
  int b0 = 0;
  size_t sm = 0;
  int nrm = 0;
  for (int q = 0; q < np; ++q) {
    const IdProb& p = ps[q];
    const int cw = ceil_div(p.nc, g[q]);
    g[q] = ceil_div(p.nc, cw);  // no CTA without columns
    parts[2 * q] = b0;
    parts[2 * q + 1] = g[q];
    b0 += g[q];
    sm = std::max(sm, (size_t(p.nr) * cw + size_t(p.nr) + 2 * size_t(cw)) * sizeof(double));
    nrm = std::max(nrm, p.nr);
  }
  *G = b0;
  *smem = sm;
  *nr_max = nrm;
  return sm <= cap;
}

void grid_id_run(const std::vector<IdProb>& ps, bool paired, const std::vector<int>& parts, int G, size_t smem,
                 int nr_max, cudaStream_t s) {
  init_smem_limits();
  auto dp = to_device_tmp(ps, s);
  auto dparts = to_device_tmp(parts, s);
  TBuf<double> pub(4 * size_t(G) + 2 * size_t(G) * nr_max, s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(G));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  {
    ProfScope pr(KC_ID, s);
    RW_CUDA(cudaLaunchKernelEx(&cfg, k_cpqr_grid, (const IdProb*)dp.p, 0, int(ps.size()), (const int*)dparts.p,
                               paired ? 1 : 0, nr_max, pub.p, id_flops_counter()));
    RW_CHECK_LAUNCH();
  }
  id_finish(dp.p, 0, ps, s);
}
}  // namespace

// Up to this many problems (with enough work between them to matter) go to
// the grid-wide factorisation, every SM working on one of them, instead of
// one thread-block cluster each.
constexpr int kGridIdProbs = 32;
constexpr double kGridIdMinWork = 32768.0;

// RW_ID_GRID=0 (diagnostics) keeps every problem on thread-block clusters.
static bool grid_id_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("RW_ID_GRID");
    return !(e && e[0] == '0');
  }();
  return on;
}

bool grid_id_fits(int nr, int nc) {
  IdProb p{};
  p.nr = nr;
  p.nc = nc;
  std::vector<int> parts;
  int G = 0, nrm = 0;
  size_t smem = 0;
  return grid_id_enabled() && double(nr) * nc >= kGridIdMinWork && grid_id_plan({p}, 200 * 1024, parts, &G, &smem, &nrm);
}

void batched_id(const std::vector<IdProb>& probs_in, cudaStream_t s, bool paired) {
  if (probs_in.empty()) return;
  // Route each problem: a thread-block cluster of CS in {1, 2, 4, 8} CTAs
  // whose shared memory holds the matrix, or the global-memory kernel.
  // Pairs (paired: problems 2i and 2i+1) share one cluster of 2 CS <= 8 CTAs
  // when both fit; otherwise they are routed one by one.  CS is the
  // smallest that holds the matrix, raised while the batch stays within
  // about two CTAs per SM and every CTA keeps at least 32 columns: a pivot
  // step's update (FP64-bound) is then shared by more SMs.
  const size_t cap = 200 * 1024;
  const int sizes[4] = {1, 2, 4, 8};
  const int nsm = sm_count();
  // RW_ID_CS_MIN (tuning): smallest cluster size tried (1, 2, 4 or 8)
  static const int q_min = [] {
    const char* e = std::getenv("RW_ID_CS_MIN");
    const int v = e ? std::atoi(e) : 1;
    return v >= 8 ? 3 : v >= 4 ? 2 : v >= 2 ? 1 : 0;
  }();
  const long long units = paired ? (long long)(probs_in.size() + 1) / 2 : (long long)probs_in.size();
  int spread_q = 0;
  while (spread_q < 3 && units * sizes[spread_q + 1] * (paired ? 2 : 1) <= 2LL * nsm) ++spread_q;
  auto fitq = [&](const IdProb& p) {
    int q = -1;
    for (int t = q_min; t < 4 && q < 0; ++t) {
      const int cw = (p.nc + sizes[t] - 1) / sizes[t];
      if (cpqr_cluster_smem(p.nr, cw, kCpqrThreads) <= cap) q = t;
    }
    if (q < 0) return -1;
    while (q < spread_q && q < 3 && p.nc >= 32 * sizes[q + 1]) ++q;
    return q;
  };
  // A few problems that do not all fit a cluster (8 CTAs, or 4 per problem
  // when paired) go to the grid-wide factorisation instead.
  if (int(probs_in.size()) <= kGridIdProbs && grid_id_enabled()) {
    double work = 0.0;
    bool fit_all = true;
    for (auto& p : probs_in) {
      work += double(p.nr) * p.nc;
      const int q = fitq(p);
      fit_all = fit_all && q >= 0 && (!paired || q <= 2);
    }
    std::vector<int> parts;
    int G = 0, nrm = 0;
    size_t smem = 0;
    if (!fit_all && work >= kGridIdMinWork && grid_id_plan(probs_in, 200 * 1024, parts, &G, &smem, &nrm)) {
      grid_id_run(probs_in, paired, parts, G, smem, nrm, s);
      return;
    }
  }
  std::vector<IdProb> grp[4], pgrp[3], gl;
  const size_t n = probs_in.size();
  for (size_t i = 0; i < n;) {
    if (paired && i + 1 < n) {
      const int qa = fitq(probs_in[i]), qb = fitq(probs_in[i + 1]);
      const int q = std::max(qa, qb);
      if (qa >= 0 && qb >= 0 && q <= 2) {
        pgrp[q].push_back(probs_in[i]);
        pgrp[q].push_back(probs_in[i + 1]);
        i += 2;
        continue;
      }
    }
    const int q = fitq(probs_in[i]);
    if (q >= 0) grp[q].push_back(probs_in[i]);
    else gl.push_back(probs_in[i]);
    ++i;
  }
  std::vector<IdProb> all;
  std::vector<int> base(4, 0), pbase(3, 0);
  for (int q = 0; q < 4; ++q) { base[q] = int(all.size()); all.insert(all.end(), grp[q].begin(), grp[q].end()); }
  for (int q = 0; q < 3; ++q) { pbase[q] = int(all.size()); all.insert(all.end(), pgrp[q].begin(), pgrp[q].end()); }
  const int gbase = int(all.size());
  all.insert(all.end(), gl.begin(), gl.end());
  init_smem_limits();
  auto dp = to_device_tmp(all, s);
  // The groups (one launch per cluster shape) are independent: all but the
  // first run on side streams forked from s and joined back, so that a
  // group of a few large problems overlaps the bulk instead of following it.
  int ngroups = int(!gl.empty());
  for (int q = 0; q < 4; ++q) ngroups += int(!grp[q].empty());
  for (int q = 0; q < 3; ++q) ngroups += int(!pgrp[q].empty());
  ForkJoin fj(s, ngroups);
  auto launch = [&](const std::vector<IdProb>& g, int b0, int CS, int pr) {
    if (g.empty()) return;
    const cudaStream_t s = fj.next();
    size_t smem = 0;
    for (auto& p : g) smem = std::max(smem, cpqr_cluster_smem(p.nr, (p.nc + CS - 1) / CS, kCpqrThreads));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(g.size() * CS));
    cfg.blockDim = dim3(kCpqrThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS * (pr ? 2 : 1);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    {
      ProfScope ps(KC_ID, s);
      RW_CUDA(cudaLaunchKernelEx(&cfg, k_cpqr_cluster, (const IdProb*)dp.p, b0, CS, pr, id_flops_counter()));
      RW_CHECK_LAUNCH();
    }
    id_finish(dp.p, b0, g, s);
  };
  for (int q = 0; q < 4; ++q) launch(grp[q], base[q], sizes[q], 0);
  for (int q = 0; q < 3; ++q) launch(pgrp[q], pbase[q], sizes[q], 1);
  if (!gl.empty()) {
    size_t gl_bytes = 0;
    for (auto& p : gl) gl_bytes = std::max(gl_bytes, size_t(p.nr) * sizeof(double));
    require(gl_bytes <= cap, "batched_id: more than 25600 feature rows");
    const cudaStream_t sg = fj.next();
    ProfScope pg(KC_ID, sg);
    k_cpqr_id<false><<<int(gl.size()), 512, gl_bytes, sg>>>(dp.p, gbase, id_flops_counter());
    RW_CHECK_LAUNCH();
  }
  fj.join();
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
void axpby(const double* x, double* y, size_t n, double a, double b, cudaStream_t s) {
  if (!n) return;
  k_axpby<<<grid_for(n), 256, 0, s>>>(x, y, n, a, b);
  RW_CHECK_LAUNCH();
}
void fill_zero(double* p, size_t n, cudaStream_t s) {
  if (!n) return;
  k_fill_zero<<<grid_for(n), 256, 0, s>>>(p, n);
  RW_CHECK_LAUNCH();
}
__global__ void k_d2bf(const double* in, __nv_bfloat16* out, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    out[i] = __double2bfloat16(in[i]);
}

void copy_d2bf(const double* in, __nv_bfloat16* out, size_t n, cudaStream_t s) {
  if (n == 0) return;
  k_d2bf<<<grid_for(n), 256, 0, s>>>(in, out, n);
  RW_CHECK_LAUNCH();
}

void copy_d2f(const double* in, float* out, size_t n, cudaStream_t s) {
  if (!n) return;
  k_d2f<<<grid_for(n), 256, 0, s>>>(in, out, n);
  RW_CHECK_LAUNCH();
}

}  // namespace rw
