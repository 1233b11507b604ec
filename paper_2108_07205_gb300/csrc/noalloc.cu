// Allocation-free variant of the HBS inverse sweep (rw_hbs_apply_inverse).
//
// Some callers cannot let this library call cudaMalloc / cudaFree during a
// solve: for example a host application whose device memory is owned by
// another framework's pool with no headroom left for outside allocations, or
// a latency-critical loop that must not let an allocation or a free
// synchronise the device.  rw_hbs_apply_inverse_noalloc serves them: every
// temporary of the sweep (the per-level skeleton vectors, the launch
// descriptors and any split-K partial sums) is carved out of the fixed
// device array below, which is part of the library image.  The caller passes
// device pointers for the input and the output, as for the regular call.
//
// Limits: RW_NOALLOC_SCRATCH_BYTES (32 MiB) of scratch per device, and at
// most 8 right-hand sides (the GEMV path of the sweep).  Every GPU that loads
// the library holds the array until the process exits.  All calls share the
// array and it keeps the last call's contents; the sweep writes every
// scratch entry before it reads it, so nothing needs clearing.  Calls whose
// executions overlap on the GPU (several streams, or several host threads)
// race on the array: order them on one stream.
#include "handles.cuh"
#include <mutex>

#define RW_NOALLOC_SCRATCH_BYTES (32u << 20)

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[RW_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up on the
// first call on each device, with that device current).
void* scratch_on_current_device() {
  int dev = 0;
  RW_CUDA(cudaGetDevice(&dev));
  rw::require(dev >= 0 && dev < kMaxDevices, "noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      throw rw::Error(RW_ERR_CUDA, std::string("cudaGetSymbolAddress(noalloc scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Arena {
  char* base;
  size_t cap, used = 0;
  template <class T>
  T* take(size_t count) {
    const size_t bytes = ((count * sizeof(T) + 255) / 256) * 256;
    rw::require(used + bytes <= cap,
                "rw_hbs_apply_inverse_noalloc: problem needs more than the " +
                    std::to_string(RW_NOALLOC_SCRATCH_BYTES >> 20) + " MiB scratch array (reduce nrhs)");
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

// The sweep's launches, level by level (same operations and order as
// Hbs::sweep_inverse), as problem lists over the per-level vectors uh, qh.
std::vector<std::vector<rw::GemvProb<double>>> sweep_stages(const rw::Hbs& H, const double* b, double* x,
                                                           const std::vector<double*>& uh,
                                                           const std::vector<double*>& qh) {
  using rw::GemvProb;
  const int L = H.L, ld = 2 * H.N;
  std::vector<std::vector<GemvProb<double>>> st;
  if (L == 0) {
    st.push_back({GemvProb<double>{H.lev[0].G.p, b, x, ld, ld, ld, ld, ld, 1.0, 0.0}});
    return st;
  }
  {
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const auto& LV = H.lev[l];
    const int K = LV.koff.back();
    std::vector<GemvProb<double>> ps;
    for (int t = 0; t < nn; ++t) {
      const auto& nd = H.node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo), k = nd.k;
      const double* in = b + 2 * nd.lo;
      ps.push_back(GemvProb<double>{LV.F.p + LV.oF[t], in, uh[l] + LV.koff[t], k, n, k, ld, K, 1.0, 0.0});
      ps.push_back(GemvProb<double>{LV.G.p + LV.oG[t], in, x + 2 * nd.lo, n, n, n, ld, ld, 1.0, 0.0});
    }
    st.push_back(std::move(ps));
  }
  for (int l = L - 1; l >= 1; --l) {
    const int h0 = 1 << l, nn = 1 << l;
    const auto& LV = H.lev[l];
    const auto& LC = H.lev[l + 1];
    const int K = LV.koff.back(), KC = LC.koff.back();
    std::vector<GemvProb<double>> ps;
    for (int t = 0; t < nn; ++t) {
      const auto& nd = H.node[h0 + t];
      const double* in = uh[l + 1] + LC.koff[2 * t];
      ps.push_back(GemvProb<double>{LV.F.p + LV.oF[t], in, uh[l] + LV.koff[t], nd.k, nd.m, nd.k, KC, K, 1.0, 0.0});
      ps.push_back(GemvProb<double>{LV.G.p + LV.oG[t], in, qh[l + 1] + LC.koff[2 * t], nd.m, nd.m, nd.m, KC, KC, 1.0, 0.0});
    }
    st.push_back(std::move(ps));
  }
  {
    const int K1 = H.lev[1].koff.back();
    st.push_back({GemvProb<double>{H.lev[0].G.p, uh[1], qh[1], K1, K1, K1, K1, K1, 1.0, 0.0}});
  }
  for (int l = 1; l <= L - 1; ++l) {
    const int h0 = 1 << l, nn = 1 << l;
    const auto& LV = H.lev[l];
    const auto& LC = H.lev[l + 1];
    const int K = LV.koff.back(), KC = LC.koff.back();
    std::vector<GemvProb<double>> ps;
    for (int t = 0; t < nn; ++t) {
      const auto& nd = H.node[h0 + t];
      ps.push_back(GemvProb<double>{LV.E.p + LV.oE[t], qh[l] + LV.koff[t], qh[l + 1] + LC.koff[2 * t], nd.m, nd.k, nd.m, K, KC, 1.0, 1.0});
    }
    st.push_back(std::move(ps));
  }
  {
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const auto& LV = H.lev[l];
    const int K = LV.koff.back();
    std::vector<GemvProb<double>> ps;
    for (int t = 0; t < nn; ++t) {
      const auto& nd = H.node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      ps.push_back(GemvProb<double>{LV.E.p + LV.oE[t], qh[l] + LV.koff[t], x + 2 * nd.lo, n, nd.k, n, K, ld, 1.0, 1.0});
    }
    st.push_back(std::move(ps));
  }
  return st;
}

size_t round256(size_t bytes) { return ((bytes + 255) / 256) * 256; }

// The whole sweep with scratch from the arena.  Every piece (per-level
// vectors, each launch's descriptors and split-K partials) is sized first and
// the total checked against the array, so a sweep that does not fit is
// refused before anything is launched or written.
void sweep_noalloc(const rw::Hbs& H, const double* b, double* x, int nrhs, Arena& ar, cudaStream_t s) {
  const int L = H.L;
  size_t need = 0;
  for (int l = 1; l <= L; ++l) need += 2 * round256(size_t(H.lev[l].koff.back()) * nrhs * sizeof(double));
  {
    const std::vector<double*> none(L + 1, nullptr);
    for (const auto& ps : sweep_stages(H, b, x, none, none)) {
      size_t db = 0, se = 0;
      rw::gemv_into_sizes(ps, nrhs, &db, &se);
      need += round256(db) + (se ? round256(se * sizeof(double)) : 0);
    }
  }
  rw::require(need <= ar.cap, "rw_hbs_apply_inverse_noalloc: the sweep needs " + std::to_string(need) +
                                  " bytes of scratch, more than the " + std::to_string(RW_NOALLOC_SCRATCH_BYTES >> 20) +
                                  " MiB scratch array (reduce nrhs)");
  std::vector<double*> uh(L + 1, nullptr), qh(L + 1, nullptr);
  for (int l = 1; l <= L; ++l) {
    const int K = H.lev[l].koff.back();
    uh[l] = ar.take<double>(size_t(K) * nrhs);
    qh[l] = ar.take<double>(size_t(K) * nrhs);
  }
  for (const auto& ps : sweep_stages(H, b, x, uh, qh)) {
    size_t db = 0, se = 0;
    rw::gemv_into_sizes(ps, nrhs, &db, &se);
    void* desc = ar.take<char>(db);
    double* sc = se ? ar.take<double>(se) : nullptr;
    rw::gemv_into(ps, nrhs, desc, sc, s);
  }
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int rw_hbs_apply_inverse_noalloc(rw_hbs_t h, int nrhs, const double* b, double* x, void* stream) {
  if (!h || !b || !x) return rw::abi_fail(RW_ERR_INVALID, "rw_hbs_apply_inverse_noalloc: null argument");
  if (nrhs < 1 || nrhs > 8)
    return rw::abi_fail(RW_ERR_INVALID, "rw_hbs_apply_inverse_noalloc: nrhs must be in 1..8");
  if (b == x) return rw::abi_fail(RW_ERR_INVALID, "rw_hbs_apply_inverse_noalloc: b and x may not alias");
  try {
    if (!is_device_pointer(b) || !is_device_pointer(x))
      throw rw::Error(RW_ERR_INVALID, "rw_hbs_apply_inverse_noalloc: b and x must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Arena ar{static_cast<char*>(scratch_on_current_device()), RW_NOALLOC_SCRATCH_BYTES};
    sweep_noalloc(h->wall.hbs, b, x, nrhs, ar, s);
    rw::abi_clear_error();
    return RW_OK;
  } catch (const rw::Error& e) {
    return rw::abi_fail(e.code, e.what());
  } catch (const std::exception& e) {
    return rw::abi_fail(RW_ERR_INVALID, e.what());
  }
}
