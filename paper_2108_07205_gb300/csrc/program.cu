// Persistent cooperative executor of GEMV programs (see program.cuh).
#include "program.cuh"
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace rw {

namespace {

constexpr int TE = 256;       // copy / fill / reduce entries per tile
constexpr int SPLIT_N = 4096; // GEMVs wider than this with few row tiles are split
constexpr int SPLIT_THIN = 256; // column chunk for wide GEMVs of thin phases
constexpr int kPrefetchChunk = 16384;

struct Bases { double* p[kMaxBases]; };

// Asks the L2 to fetch phase p's matrices (bulk prefetch, no registers or
// shared memory held): every thread of the grid issues at most a few ranges.
__device__ __forceinline__ void prefetch_phase(const char* const* addr, const int* bytes, const int* off, int p) {
  const int n0 = off[p], n1 = off[p + 1];
  // ranges dealt round-robin over the CTAs first, then over their threads
  const int gt = blockIdx.x + gridDim.x * threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int i = n0 + gt; i < n1; i += gs)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(addr[i]), "r"(bytes[i]) : "memory");
}

template <int NR, int TR>
__device__ void do_gemv(const GOp& o, int tile, const Bases& B, int r0, double (*xs)[NR], double (*red)[TR][NR]) {
  // 256 threads = TR rows x LANES column lanes; each lane keeps UNR
  // independent accumulator chains per right-hand side
  constexpr int LANES = 256 / TR;
  const int lr = threadIdx.x % TR, lc = threadIdx.x / TR;
  const int row = tile * TR + lr;
  const double* x = B.p[o.xb] + o.xo + size_t(r0) * o.ldx;
  double* y = B.p[o.yb] + o.yo + size_t(r0) * o.ldy;
  // UNR independent chains per right-hand side (UNR * NR = 16 accumulators)
  constexpr int UNR = NR == 1 ? 16 : NR == 2 ? 8 : NR <= 4 ? 4 : 2;
  double acc[UNR][NR];
#pragma unroll
  for (int u = 0; u < UNR; ++u)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[u][r] = 0.0;
  for (int cb = 0; cb < o.n; cb += 256) {
    const int ncur = min(256, o.n - cb);
    __syncthreads();
    for (int e = threadIdx.x; e < ncur; e += 256)
#pragma unroll
      for (int r = 0; r < NR; ++r) xs[e][r] = x[cb + e + size_t(r) * o.ldx];
    __syncthreads();
    if (row < o.m) {
      const double* a = o.A + row + size_t(cb) * o.lda;
      int j = lc;
      for (; j + LANES * (UNR - 1) < ncur; j += LANES * UNR) {
        double v[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) v[u] = a[size_t(j + LANES * u) * o.lda];
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
          for (int r = 0; r < NR; ++r) acc[u][r] = fma(v[u], xs[j + LANES * u][r], acc[u][r]);
      }
      for (; j < ncur; j += LANES) {
        const double v = a[size_t(j) * o.lda];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[0][r] = fma(v, xs[j][r], acc[0][r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < UNR; ++u) s += acc[u][r];
    red[lc][lr][r] = s;
  }
  __syncthreads();
  if (lc == 0 && row < o.m) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < LANES; ++q) s += red[q][lr][r];
      double* yp = y + row + size_t(r) * o.ldy;
      double v = o.alpha * s;
      if (o.beta != 0.0) v += o.beta * *yp;
      *yp = v;
    }
  }
  __syncthreads();
}

template <int NR, int TR>
__global__ void __launch_bounds__(256, 2) k_program(const GOp* ops, const int* tile0, const int* tile_op, const int* phase, int nphases,
                                                 Bases B, int r0, const char* const* pf_addr, const int* pf_bytes,
                                                 const int* pf_off, int pf_mode, long long* ptimes) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double xs[256][NR];
  __shared__ double red[256 / TR][TR][NR];
  if (ptimes && blockIdx.x == 0 && threadIdx.x == 0) ptimes[0] = clock64();
  if (pf_mode == 1) prefetch_phase(pf_addr, pf_bytes, pf_off, 0);
  for (int ph = 0; ph < nphases; ++ph) {
    // the next phase's matrices stream into L2 while this phase runs
    if (pf_mode && ph + 1 < nphases) prefetch_phase(pf_addr, pf_bytes, pf_off, ph + 1);
    const int o0 = phase[ph], o1 = phase[ph + 1];
    const int t0 = tile0[o0], t1 = tile0[o1];
    for (int t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
      const int lo = tile_op[t];  // op with tile0[op] <= t < tile0[op + 1]
      const GOp& o = ops[lo];
      const int tile = t - tile0[lo];
      if (o.kind == OP_GEMV) {
        do_gemv<NR, TR>(o, tile, B, r0, xs, red);
      } else {
        const int i = tile * TE + threadIdx.x;
        if (i < o.m) {
          const double* x = (o.kind == OP_ZERO) ? nullptr : B.p[o.xb] + o.xo + size_t(r0) * o.ldx;
          double* y = B.p[o.yb] + o.yo + size_t(r0) * o.ldy;
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            if (o.kind == OP_COPY) {
              y[(o.iy ? o.iy[i] : i) + size_t(r) * o.ldy] = x[(o.ix ? o.ix[i] : i) + size_t(r) * o.ldx];
            } else if (o.kind == OP_ZERO) {
              y[(o.iy ? o.iy[i] : i) + size_t(r) * o.ldy] = 0.0;
            } else {  // REDUCE: parts are m apart in x
              double s = 0.0;
              for (int q = 0; q < o.n; ++q) s += x[i + size_t(q) * o.m + size_t(r) * o.ldx];
              double* yp = y + i + size_t(r) * o.ldy;
              double v = o.alpha * s;
              if (o.beta != 0.0) v += o.beta * *yp;
              *yp = v;
            }
          }
        }
      }
    }
    grid.sync();
    if (ptimes && blockIdx.x == 0 && threadIdx.x == 0) ptimes[ph + 1] = clock64();
  }
}

template <int TR>
const void* kernel_ptr(int nr) {
  switch (nr) {
    case 1: return reinterpret_cast<const void*>(&k_program<1, TR>);
    case 2: return reinterpret_cast<const void*>(&k_program<2, TR>);
    case 3: return reinterpret_cast<const void*>(&k_program<3, TR>);
    case 4: return reinterpret_cast<const void*>(&k_program<4, TR>);
    case 5: return reinterpret_cast<const void*>(&k_program<5, TR>);
    case 6: return reinterpret_cast<const void*>(&k_program<6, TR>);
    case 7: return reinterpret_cast<const void*>(&k_program<7, TR>);
    default: return reinterpret_cast<const void*>(&k_program<8, TR>);
  }
}

const void* kernel_for(int tr, int nr) {
  return tr == 16 ? kernel_ptr<16>(nr) : tr == 64 ? kernel_ptr<64>(nr) : kernel_ptr<32>(nr);
}

int host_tiles(const GOp& o, int tr) { return o.kind == OP_GEMV ? (o.m + tr - 1) / tr : (o.m + TE - 1) / TE; }

}  // namespace

// RW_PROG_PREFETCH (tuning): 0 = no L2 prefetch, 1 = every phase including
// the first, 2 = the phases after the first (default)
static int prefetch_mode() {
  static const int m = [] {
    const char* e = std::getenv("RW_PROG_PREFETCH");
    return e ? std::atoi(e) : 2;
  }();
  return m;
}

// RW_PROG_TIMES=1 (diagnostics): print each phase's duration in cycles after
// every run (synchronises the stream)
static bool phase_times() {
  static const bool on = [] {
    const char* e = std::getenv("RW_PROG_TIMES");
    return e && e[0] == '1';
  }();
  return on;
}

static std::vector<GOp>& phase_at(std::vector<std::vector<GOp>>& ph, int p) {
  if (int(ph.size()) <= p) ph.resize(p + 1);
  return ph[p];
}

void Program::gemv(int p, const double* A, int m, int n, int lda, int xb, long long xo, int ldx, int yb,
                   long long yo, int ldy, double alpha, double beta) {
  if (m <= 0) return;
  GOp o{};
  o.kind = OP_GEMV;
  o.m = m; o.n = n; o.A = A; o.lda = lda;
  o.xb = xb; o.xo = xo; o.ldx = ldx; o.yb = yb; o.yo = yo; o.ldy = ldy;
  o.alpha = alpha; o.beta = beta;
  phase_at(phases_, p).push_back(o);
  mat_elems_ += (long long)m * n;
}

void Program::copy(int p, int n, int xb, long long xo, int ldx, const int* ix, int yb, long long yo, int ldy,
                   const int* iy) {
  if (n <= 0) return;
  GOp o{};
  o.kind = OP_COPY;
  o.m = n; o.xb = xb; o.xo = xo; o.ldx = ldx; o.ix = ix; o.yb = yb; o.yo = yo; o.ldy = ldy; o.iy = iy;
  phase_at(phases_, p).push_back(o);
}

void Program::zero(int p, int n, int yb, long long yo, int ldy, const int* iy) {
  if (n <= 0) return;
  GOp o{};
  o.kind = OP_ZERO;
  o.m = n; o.yb = yb; o.yo = yo; o.ldy = ldy; o.iy = iy;
  phase_at(phases_, p).push_back(o);
}

long long Program::ws_alloc(long long elems) {
  const long long o = ws_;
  ws_ += (elems + 31) / 32 * 32;
  return o;
}

void Program::finalize(cudaStream_t s) {
  // split wide GEMVs (few row tiles, many columns) into column-chunk partial
  // products in the workspace and a reduce op in an extra phase
  // wide GEMVs in phases with fewer row tiles than SMs (one SM would run a
  // whole wide tile at its FP64 rate) are split into column chunks of
  // SPLIT_THIN as well
  std::vector<std::vector<GOp>> out;
  const int wsb = 2;  // workspace base index (by convention)
  int nsm0 = 0, dev0 = 0;
  RW_CUDA(cudaGetDevice(&dev0));
  RW_CUDA(cudaDeviceGetAttribute(&nsm0, cudaDevAttrMultiProcessorCount, dev0));
  for (auto& ph : phases_) {
    std::vector<GOp> cur, red;
    int t32 = 0;
    for (const GOp& o : ph) t32 += host_tiles(o, 32);
    const bool thin = t32 < nsm0;
    for (const GOp& o : ph) {
      const bool wide = o.kind == OP_GEMV && o.n > SPLIT_N && host_tiles(o, 32) < 38;
      const bool thin_wide = o.kind == OP_GEMV && thin && o.n >= 2 * SPLIT_THIN;
      if (wide || thin_wide) {
        const int chunk = wide ? SPLIT_N : std::max(SPLIT_THIN, (o.n + 7) / 8);
        const int parts = (o.n + chunk - 1) / chunk;
        const long long pw = ws_alloc((long long)parts * o.m);
        for (int q = 0; q < parts; ++q) {
          GOp g = o;
          const int c0 = q * chunk, c1 = std::min(o.n, c0 + chunk);
          g.A = o.A + size_t(c0) * o.lda;
          g.n = c1 - c0;
          g.xo = o.xo + c0;
          g.yb = wsb; g.yo = pw + (long long)q * o.m; g.ldy = -1;  // ld patched at run (workspace ld)
          g.alpha = 1.0; g.beta = 0.0;
          cur.push_back(g);
        }
        GOp r{};
        r.kind = OP_REDUCE;
        r.m = o.m; r.n = parts;
        r.xb = wsb; r.xo = pw; r.ldx = -1;
        r.yb = o.yb; r.yo = o.yo; r.ldy = o.ldy;
        r.alpha = o.alpha; r.beta = o.beta;
        red.push_back(r);
      } else {
        cur.push_back(o);
      }
    }
    out.push_back(cur);
    if (!red.empty()) out.push_back(red);
  }
  // workspace leading dimension: the per-RHS block size
  for (auto& ph : out)
    for (GOp& o : ph) {
      if (o.ldx == -1) o.ldx = int(ws_);
      if (o.ldy == -1) o.ldy = int(ws_);
    }
  std::vector<GOp> flat;
  std::vector<int> phase(1, 0);
  for (auto& ph : out) {
    for (const GOp& o : ph) flat.push_back(o);
    phase.push_back(int(flat.size()));
  }
  nph_ = int(out.size());
  if (phase_times()) {
    for (size_t q = 0; q < out.size(); ++q) {
      long long ent = 0;
      int ng = 0, t32 = 0, mm = 0, mn = 0;
      for (const GOp& o : out[q]) {
        t32 += host_tiles(o, 32);
        if (o.kind != OP_GEMV) continue;
        ++ng;
        ent += (long long)o.m * o.n;
        mm = std::max(mm, o.m);
        mn = std::max(mn, o.n);
      }
      std::fprintf(stderr, "[rw program] phase %zu: %zu ops (%d GEMV), %d tiles of 32, max %d x %d, %lld entries\n", q,
                   out[q].size(), ng, t32, mm, mn, ent);
    }
  }
  d_ops_ = to_device(flat, s);
  d_phase_ = to_device(phase, s);
  {
    // prefetch ranges: the span of each GEMV's matrix, cut into chunks whose
    // ends are rounded down to 16 bytes (so every range stays inside the
    // matrix's allocation)
    std::vector<const char*> pa;
    std::vector<int> pb, po(1, 0);
    for (auto& ph : out) {
      for (const GOp& o : ph) {
        if (o.kind != OP_GEMV || o.m <= 0 || o.n <= 0) continue;
        const uintptr_t b0 = reinterpret_cast<uintptr_t>(o.A);
        const uintptr_t b1 = b0 + (size_t(o.lda) * (o.n - 1) + o.m) * sizeof(double);
        uintptr_t a = b0 & ~uintptr_t(15);
        const uintptr_t e = b1 & ~uintptr_t(15);
        while (a < e) {
          const uintptr_t c = std::min<uintptr_t>(e, a + kPrefetchChunk);
          pa.push_back(reinterpret_cast<const char*>(a));
          pb.push_back(int(c - a));
          a = c;
        }
      }
      po.push_back(int(pa.size()));
    }
    if (pa.empty()) { pa.push_back(nullptr); pb.push_back(0); }
    d_pf_addr_ = to_device(pa, s);
    d_pf_bytes_ = to_device(pb, s);
    d_pf_off_ = to_device(po, s);
  }
  int dev = 0, nsm = 0;
  RW_CUDA(cudaGetDevice(&dev));
  RW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int trs[3] = {16, 32, 64};
  for (int v = 0; v < 3; ++v) {
    std::vector<int> tile0(1, 0);
    int maxt = 1;
    size_t o0 = 0;
    for (auto& ph : out) {
      int tph = 0;
      for (const GOp& o : ph) {
        const int t = host_tiles(o, trs[v]);
        tph += t;
        tile0.push_back(tile0.back() + t);
      }
      maxt = std::max(maxt, tph);
      o0 += ph.size();
    }
    d_tile_[v] = to_device(tile0, s);
    std::vector<int> top(std::max(tile0.back(), 1), 0);
    for (size_t q = 0; q + 1 < tile0.size(); ++q)
      for (int t = tile0[q]; t < tile0[q + 1]; ++t) top[t] = int(q);
    d_top_[v] = to_device(top, s);
    int per = 0;
    RW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel_for(trs[v], 8), 256, 0));
    grid_[v] = std::max(1, std::min(maxt, nsm * std::max(per, 1)));
  }
  RW_CUDA(cudaStreamSynchronize(s));
}

void Program::run(double* const* bases, int nrhs, cudaStream_t s) const {
  if (nph_ == 0) return;
  Bases B;
  for (int i = 0; i < kMaxBases; ++i) B.p[i] = bases[i];
  const int v = tr_index_;
  const int trs[3] = {16, 32, 64};
  const GOp* ops = d_ops_.p;
  const int* t0 = d_tile_[v].p;
  const int* top = d_top_[v].p;
  const int* ph = d_phase_.p;
  int nphases = nph_;
  TBuf<long long> times(phase_times() ? size_t(nph_ + 1) : 0, s);
  for (int r0 = 0; r0 < nrhs; r0 += 8) {
    const int nr = std::min(8, nrhs - r0);
    const char* const* pfa = d_pf_addr_.p;
    const int* pfb = d_pf_bytes_.p;
    const int* pfo = d_pf_off_.p;
    int pfm = prefetch_mode();
    long long* pt = phase_times() ? times.p : nullptr;
    void* args[] = {(void*)&ops, (void*)&t0, (void*)&top, (void*)&ph, (void*)&nphases, (void*)&B, (void*)&r0,
                    (void*)&pfa, (void*)&pfb, (void*)&pfo, (void*)&pfm, (void*)&pt};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_[v]);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ProfScope prof(KC_GEMV, s, 0.0, 0.0);
    RW_CUDA(cudaLaunchKernelExC(&cfg, kernel_for(trs[v], nr), args));
    RW_CHECK_LAUNCH();
    if (phase_times()) {
      // diagnostics: cycles of each phase as seen by CTA 0 (its SM's clock)
      std::vector<long long> h(nph_ + 1);
      RW_CUDA(cudaMemcpyAsync(h.data(), times.p, h.size() * sizeof(long long), cudaMemcpyDeviceToHost, s));
      RW_CUDA(cudaStreamSynchronize(s));
      std::fprintf(stderr, "[rw program] %d phases, grid %d, TR %d:", nph_, grid_[v], trs[v]);
      for (int q = 0; q < nph_; ++q) std::fprintf(stderr, " %lld", h[q + 1] - h[q]);
      std::fprintf(stderr, " cycles\n");
    }
  }
}

float Program::autotune(double* const* bases, int nrhs, cudaStream_t s) {
  // time each tile height (best of 3 after one warm-up run) and keep the fastest
  cudaEvent_t a, b;
  RW_CUDA(cudaEventCreate(&a));
  RW_CUDA(cudaEventCreate(&b));
  float best = 1e30f;
  int bestv = 1;
  for (int v = 0; v < 3; ++v) {
    tr_index_ = v;
    run(bases, nrhs, s);
    float tmin = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      RW_CUDA(cudaEventRecord(a, s));
      run(bases, nrhs, s);
      RW_CUDA(cudaEventRecord(b, s));
      RW_CUDA(cudaEventSynchronize(b));
      float ms = 0.f;
      RW_CUDA(cudaEventElapsedTime(&ms, a, b));
      tmin = std::min(tmin, ms);
    }
    if (tmin < best) { best = tmin; bestv = v; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  tr_index_ = bestv;
  return best;
}

}  // namespace rw
