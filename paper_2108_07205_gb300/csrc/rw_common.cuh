// Shared declarations of the rwsolve CUDA library: error handling, device
// buffers, node sets and the Stokes kernel entries of Sec. 2.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <stdexcept>

#include "../../include/rwsolve.h"

namespace rw {

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define RW_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      throw ::rw::Error(RW_ERR_CUDA, std::string(#call) + ": " +             \
                                         cudaGetErrorString(e_));            \
  } while (0)

// Every kernel launch site ends with RW_CHECK_LAUNCH(), which also counts it.
extern std::atomic<unsigned long long> g_launches;
#define RW_CHECK_LAUNCH()                                              \
  do {                                                                 \
    ::rw::g_launches.fetch_add(1, std::memory_order_relaxed);          \
    RW_CUDA(cudaGetLastError());                                       \
  } while (0)

inline void require(bool ok, const std::string& msg, int code = RW_ERR_INVALID) {
  if (!ok) throw Error(code, msg);
}

// ---------------------------------------------------------------- memory
// Allocation stream of the calling host thread: when set, DBuf allocations
// are stream ordered on it (cudaMallocAsync / cudaFreeAsync), so freeing a
// handle's memory does not synchronise the whole device.  Unset (the
// default), DBuf uses cudaMalloc / cudaFree.
extern thread_local cudaStream_t tl_alloc_stream;
// Once per device, before its first stream-ordered allocation: the default
// memory pool keeps freed memory (up to a quarter of the device, or
// RW_POOL_RETAIN_BYTES) instead of returning it to the driver at every
// synchronisation, so a refinement's temporaries and factors are recycled
// from one time step to the next instead of being mapped afresh.
void pool_retain_once();
// Fork-join over side streams of the calling host thread (up to 7, created
// on first use and kept for the thread's lifetime): next() returns the
// caller's stream s first, then side streams that wait for the work queued
// on s so far; join() (or the destructor) makes s wait for every side stream
// handed out.  With n <= 1 everything stays on s.
class ForkJoin {
 public:
  ForkJoin(cudaStream_t s, int n);
  ForkJoin(const ForkJoin&) = delete;
  ForkJoin& operator=(const ForkJoin&) = delete;
  cudaStream_t next();
  void join();
  ~ForkJoin();

 private:
  cudaStream_t s_;
  int n_, used_ = 0;
  bool joined_ = false;
};

struct AllocStreamScope {
  cudaStream_t prev;
  explicit AllocStreamScope(cudaStream_t s) : prev(tl_alloc_stream) { tl_alloc_stream = s; }
  ~AllocStreamScope() { tl_alloc_stream = prev; }
};

// Owning device buffer.  Moves only.
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t as = nullptr;
  bool async = false;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), as(o.as), async(o.async) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; as = o.as; async = o.async; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    n = count;
    if (count) {
      cudaError_t e;
      if (tl_alloc_stream) {
        as = tl_alloc_stream;
        async = true;
        pool_retain_once();
        e = cudaMallocAsync(reinterpret_cast<void**>(&p), count * sizeof(T), as);
      } else {
        async = false;
        e = cudaMalloc(&p, count * sizeof(T));
      }
      if (e != cudaSuccess) {
        p = nullptr; n = 0;
        throw Error(RW_ERR_OOM, std::string("device allocation: ") + cudaGetErrorString(e));
      }
    }
  }
  void release() {
    if (p) {
      if (async) cudaFreeAsync(p, as); else cudaFree(p);
    }
    p = nullptr; n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
  void upload(const std::vector<T>& h, cudaStream_t s) {
    if (h.size() != n) alloc(h.size());
    if (n) RW_CUDA(cudaMemcpyAsync(p, h.data(), bytes(), cudaMemcpyHostToDevice, s));
  }
  std::vector<T> download(cudaStream_t s) const {
    std::vector<T> h(n);
    if (n) {
      RW_CUDA(cudaMemcpyAsync(h.data(), p, bytes(), cudaMemcpyDeviceToHost, s));
      RW_CUDA(cudaStreamSynchronize(s));
    }
    return h;
  }
  void zero(cudaStream_t s) { if (n) RW_CUDA(cudaMemsetAsync(p, 0, bytes(), s)); }
};

// Stream-ordered temporary (cudaMallocAsync / cudaFreeAsync): no implicit
// device synchronisation when it is released.
template <class T>
struct TBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  TBuf() = default;
  TBuf(size_t count, cudaStream_t st) : s(st) {
    n = count;
    if (count) {
      pool_retain_once();
      cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&p), count * sizeof(T), st);
      if (e != cudaSuccess) {
        p = nullptr; n = 0;
        throw Error(RW_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
      }
    }
  }
  TBuf(const TBuf&) = delete;
  TBuf& operator=(const TBuf&) = delete;
  TBuf(TBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
  TBuf& operator=(TBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~TBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr; n = 0;
  }
};

template <class T>
TBuf<T> to_device_tmp(const std::vector<T>& h, cudaStream_t s) {
  TBuf<T> d(h.size(), s);
  if (h.size()) RW_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return d;
}

template <class T>
DBuf<T> to_device(const std::vector<T>& h, cudaStream_t s) {
  DBuf<T> d(h.size());
  if (h.size()) RW_CUDA(cudaMemcpyAsync(d.p, h.data(), d.bytes(), cudaMemcpyHostToDevice, s));
  return d;
}

// ---------------------------------------------------------------- nodes
// Curve description on the device (RW_CURVE_* and its parameters).
struct Curve {
  int kind;
  double p[8];
};

// Structure-of-arrays view of a node set on the device: position, outward
// normal, smooth quadrature weight and signed curvature per point.  kind 0 is
// a wall (double layer with the N term of Remark 2.1); kind 1 is a hole
// carrying the combined field D + S of Eq. exterior_BIE (App. B); kind 2 is
// an exterior wall (Sec. 2.2: 1/2 I + D + S on one closed curve), whose
// single layer takes a singular rule on the panels next to each target and
// needs, per node, its parameter t and its panel's midpoint tm and
// half-width th in t, plus the curve itself.
struct NodesView {
  const double *x, *y, *nx, *ny, *w, *kappa;
  int n;
  int kind;
  const double *t, *tm, *th;  // kind 2 only (else null)
  Curve curve;                // kind 2 only
};

constexpr int kNodesExterior = 2;  // NodesView::kind of an exterior wall

struct Nodes {
  DBuf<double> buf;   // 6 x n column-major: x, y, nx, ny, w, kappa
  DBuf<double> pbuf;  // kind 2: 3 x n column-major: t, tm, th
  int n = 0;
  int kind = 0;       // NodesView::kind
  Curve curve{};      // kind 2
  std::vector<double> hx, hy;       // host copy of positions (planning only)
  std::vector<double> ht, htm, hth; // kind 2: host copy of t, tm, th
  void alloc(int count) { n = count; buf.alloc(size_t(6) * count); }
  NodesView view() const {
    const double* b = buf.p;
    const double* q = kind == kNodesExterior ? pbuf.p : nullptr;
    return NodesView{b, b + n, b + 2 * size_t(n), b + 3 * size_t(n),
                     b + 4 * size_t(n), b + 5 * size_t(n), n, kind,
                     q, q ? q + n : nullptr, q ? q + 2 * size_t(n) : nullptr, curve};
  }
};

constexpr double kPi = 3.141592653589793238462643383279502884;

// ---------------------------------------------------------------- stream
struct StreamGuard {
  cudaStream_t s;
  explicit StreamGuard(void* p) : s(static_cast<cudaStream_t>(p)) {}
};

inline int ceil_div(long long a, long long b) { return int((a + b - 1) / b); }

// Opt-in kernel profiler (rw_profile / rw_profile_read): when enabled, each
// launch site records CUDA events on its own stream around its launches and
// adds its algorithmic flops and bytes to a per-class total.
enum KClass { KC_ID = 0, KC_GEMM, KC_GEMV, KC_INVERSE, KC_EVAL, KC_OTHER, KC_GEMM_F32, KC_GEMM_DF, KC_COUNT };
bool prof_enabled();
struct ProfScope {
  bool on;
  int cls;
  cudaStream_t s;
  double flops, bytes;
  cudaEvent_t a = nullptr;
  ProfScope(int cls_, cudaStream_t st, double fl = 0.0, double by = 0.0);
  ~ProfScope();
};
// Device counter of column-pivoted QR flops (added by the kernels).
double* id_flops_counter();
void profile_enable(bool on);
void profile_read(long long* launches, double* ms, double* flops, double* bytes);

// Phase timer for the refinement and build (enabled by RW_TRACE=1): prints
// wall-clock time per phase, synchronising the stream at each mark.
struct Trace {
  cudaStream_t s;
  bool on;
  double t0;
  const char* what;
  explicit Trace(cudaStream_t st, const char* w);
  void mark(const char* phase);
};

}  // namespace rw
