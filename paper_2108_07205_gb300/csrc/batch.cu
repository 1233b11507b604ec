// Batched solve of many refined walls: the direct
// solves of n refinements, each on its own wall, are merged into one GEMV
// program (phases aligned by index: scatter, sweeps leaf to root to leaf,
// Woodbury, gather) and executed by one persistent cooperative launch per 8
// right-hand sides, optionally replayed from a captured CUDA graph.  The
// GEMV tile height is chosen by an autotuner (timing 16/32/64-row tiles on
// the batch itself), with an optional on-disk cache (RW_AUTOTUNE_CACHE).
#include "handles.cuh"
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <sstream>

struct rw_batch_s {
  std::vector<const rw::Refinement*> refs;
  std::vector<long long> off;  // row offsets of each instance (size n + 1)
  rw::Program prog;
  // iterative refinement (built on first use): ext-space offsets of the
  // instances, the programs g_n -> g_ext, direct solve, operator, x_ext ->
  // tau_n, and their buffers
  bool ir_built = false;
  std::vector<long long> eoff;
  rw::Program p_in, p_dir, p_op, p_out;
  rw::DBuf<long long> d_eoff;
  rw::DBuf<double> ws_ir, gx, xx, rx, dx, dots;
  rw::DBuf<double> ws, gbuf, tbuf;
  std::map<int, cudaGraphExec_t> graphs;  // per nrhs
  std::string key;
  cudaStream_t cs = nullptr;             // capture / replay stream (the caller's
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;  // stream may be the legacy one)
  ~rw_batch_s() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    if (cs) { cudaStreamSynchronize(cs); cudaStreamDestroy(cs); }
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
  }
};

namespace {

bool is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// out[i * nrhs + r] = sum over the rows of instance i of a[row, r] b[row, r]
// (one CTA per instance and right-hand side, fixed-order reduction).
__global__ void k_seg_dots(const double* a, const double* b, long long ld, const long long* seg, int nrhs,
                           double* out) {
  const int i = blockIdx.x, r = blockIdx.y;
  const double* ar = a + size_t(r) * ld;
  const double* br = b + size_t(r) * ld;
  double s = 0.0;
  for (long long q = seg[i] + threadIdx.x; q < seg[i + 1]; q += blockDim.x) s += ar[q] * br[q];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[size_t(i) * nrhs + r] = red[0];
}

void build_ir(rw_batch_s* b, cudaStream_t s) {
  const int n = int(b->refs.size());
  b->eoff.assign(1, 0);
  for (const rw::Refinement* f : b->refs) b->eoff.push_back(b->eoff.back() + 2LL * (f->No + f->Np));
  const long long E = b->eoff.back(), G = b->off.back();
  if (E >= (1LL << 31)) throw rw::Error(RW_ERR_INVALID, "rw_batch_solve_ir: batch too large");
  for (int i = 0; i < n; ++i) {
    const rw::Refinement* f = b->refs[i];
    f->emit_to_ext(b->p_in, 0, b->off[i], int(G), 1, b->eoff[i], int(E));
    f->emit_ext_direct(b->p_dir, 0, b->eoff[i], int(E), 1, b->eoff[i], int(E));
    f->emit_ext_operator(b->p_op, 0, b->eoff[i], int(E), 1, b->eoff[i], int(E));
    f->emit_from_ext(b->p_out, 0, b->eoff[i], int(E), 1, b->off[i], int(G));
  }
  for (rw::Program* P : {&b->p_in, &b->p_dir, &b->p_op, &b->p_out}) {
    P->set_tile_rows(b->prog.tile_rows());
    P->finalize(s);
  }
  b->d_eoff = rw::to_device(b->eoff, s);
  RW_CUDA(cudaStreamSynchronize(s));
  b->ir_built = true;
}

void ensure(rw_batch_s* b, int nrhs) {
  const size_t rows = size_t(b->off.back());
  const size_t need_ws = size_t(std::max<long long>(b->prog.ws_per_rhs(), 1)) * nrhs;
  if (b->ws.n < need_ws) b->ws.alloc(need_ws);
  if (b->gbuf.n < rows * nrhs) { b->gbuf.alloc(rows * nrhs); b->tbuf.alloc(rows * nrhs); }
}

int cached_tile_rows(const std::string& key) {
  const char* path = std::getenv("RW_AUTOTUNE_CACHE");
  if (!path) return 0;
  std::ifstream in(path);
  std::string k;
  int tr;
  while (in >> k >> tr)
    if (k == key) return tr;
  return 0;
}

void store_tile_rows(const std::string& key, int tr) {
  const char* path = std::getenv("RW_AUTOTUNE_CACHE");
  if (!path) return;
  std::ofstream out(path, std::ios::app);
  out << key << " " << tr << "\n";
}

}  // namespace

extern "C" {

int rw_batch_create(int n, const rw_ref_t* refs, void* stream, rw_batch_t* out) {
  if (n < 1 || !refs || !out) return rw::abi_fail(RW_ERR_INVALID, "rw_batch_create: bad argument");
  *out = nullptr;
  auto* b = new rw_batch_s;
  try {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    b->off.push_back(0);
    for (int i = 0; i < n; ++i) {
      if (!refs[i]) throw rw::Error(RW_ERR_INVALID, "rw_batch_create: null refinement");
      b->refs.push_back(&refs[i]->ref);
      b->off.push_back(b->off.back() + 2LL * refs[i]->ref.Nn);
    }
    const long long G = b->off.back();
    if (G >= (1LL << 31)) throw rw::Error(RW_ERR_INVALID, "rw_batch_create: batch too large");
    // bases: 0 = g (G x nrhs), 1 = tau (G x nrhs), 2 = workspace
    for (int i = 0; i < n; ++i) b->refs[i]->emit_solve(b->prog, 0, b->off[i], int(G), 1, b->off[i], int(G));
    b->prog.finalize(s);
    std::ostringstream k;
    k << "batch-n" << n << "-rows" << G << "-ops" << b->prog.matrix_elems();
    b->key = k.str();
    const int tr = cached_tile_rows(b->key);
    if (tr) b->prog.set_tile_rows(tr);
  } catch (const rw::Error& e) {
    delete b;
    return rw::abi_fail(e.code, e.what());
  } catch (const std::exception& e) {
    delete b;
    return rw::abi_fail(RW_ERR_INVALID, e.what());
  }
  *out = b;
  rw::abi_clear_error();
  return RW_OK;
}

int rw_batch_rows(rw_batch_t b, long long* offsets) {
  if (!b || !offsets) return rw::abi_fail(RW_ERR_INVALID, "rw_batch_rows: bad argument");
  for (size_t i = 0; i < b->off.size(); ++i) offsets[i] = b->off[i];
  return RW_OK;
}

int rw_batch_autotune(rw_batch_t b, int nrhs, void* stream, int* tile_rows, float* ms) {
  if (!b || nrhs < 1 || nrhs > 8) return rw::abi_fail(RW_ERR_INVALID, "rw_batch_autotune: nrhs must be in 1..8");
  try {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ensure(b, nrhs);
    RW_CUDA(cudaMemsetAsync(b->gbuf.p, 0, b->gbuf.bytes(), s));
    double* bases[rw::kMaxBases] = {b->gbuf.p, b->tbuf.p, b->ws.p, nullptr};
    const float t = b->prog.autotune(bases, nrhs, s);
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    store_tile_rows(b->key, b->prog.tile_rows());
    if (tile_rows) *tile_rows = b->prog.tile_rows();
    if (ms) *ms = t;
  } catch (const rw::Error& e) {
    return rw::abi_fail(e.code, e.what());
  }
  rw::abi_clear_error();
  return RW_OK;
}

int rw_batch_solve(rw_batch_t b, int nrhs, const double* g, double* tau, int use_graph, void* stream) {
  if (!b || !g || !tau || nrhs < 1) return rw::abi_fail(RW_ERR_INVALID, "rw_batch_solve: bad argument");
  for (const rw::Refinement* f : b->refs)
    if (f->wall->opts.mixed_factor)
      return rw::abi_fail(RW_ERR_INVALID, "rw_batch_solve: the direct batch solve needs FP64 factorisations; a "
                                          "refinement whose X is not FP64 (opts.mixed_factor) takes rw_batch_solve_ir");
  try {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ensure(b, nrhs);
    const size_t bytes = size_t(b->off.back()) * nrhs * sizeof(double);
    const bool gdev = is_dev(g), tdev = is_dev(tau);
    RW_CUDA(cudaMemcpyAsync(b->gbuf.p, g, bytes, gdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    double* bases[rw::kMaxBases] = {b->gbuf.p, b->tbuf.p, b->ws.p, nullptr};
    if (use_graph) {
      if (!b->cs) {
        RW_CUDA(cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking));
        RW_CUDA(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
        RW_CUDA(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
      }
      auto it = b->graphs.find(nrhs);
      if (it == b->graphs.end()) {
        cudaGraph_t graph = nullptr;
        RW_CUDA(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
        try {
          b->prog.run(bases, nrhs, b->cs);
        } catch (...) {
          cudaStreamEndCapture(b->cs, &graph);
          if (graph) cudaGraphDestroy(graph);
          throw;
        }
        RW_CUDA(cudaStreamEndCapture(b->cs, &graph));
        cudaGraphExec_t exec;
        const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        RW_CUDA(e);
        it = b->graphs.emplace(nrhs, exec).first;
      }
      RW_CUDA(cudaEventRecord(b->ev_in, s));
      RW_CUDA(cudaStreamWaitEvent(b->cs, b->ev_in, 0));
      RW_CUDA(cudaGraphLaunch(it->second, b->cs));
      RW_CUDA(cudaEventRecord(b->ev_out, b->cs));
      RW_CUDA(cudaStreamWaitEvent(s, b->ev_out, 0));
    } else {
      b->prog.run(bases, nrhs, s);
    }
    RW_CUDA(cudaMemcpyAsync(tau, b->tbuf.p, bytes, tdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!tdev || !gdev) RW_CUDA(cudaStreamSynchronize(s));
  } catch (const rw::Error& e) {
    return rw::abi_fail(e.code, e.what());
  }
  rw::abi_clear_error();
  return RW_OK;
}

int rw_batch_solve_ir(rw_batch_t b, int nrhs, const double* g, double* tau, double tol, int maxit, void* stream,
                      int* iters, double* relres) {
  if (!b || !g || !tau || nrhs < 1 || !(tol > 0.0) || maxit < 0)
    return rw::abi_fail(RW_ERR_INVALID, "rw_batch_solve_ir: bad argument");
  int it = 0;
  double worst = 0.0;
  try {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!b->ir_built) build_ir(b, s);
    const int n = int(b->refs.size());
    const long long G = b->off.back(), E = b->eoff.back();
    long long wsn = 1;
    for (const rw::Program* P : {&b->p_in, &b->p_dir, &b->p_op, &b->p_out}) wsn = std::max(wsn, P->ws_per_rhs());
    if (b->ws_ir.n < size_t(wsn) * nrhs) b->ws_ir.alloc(size_t(wsn) * nrhs);
    if (b->gx.n < size_t(E) * nrhs) {
      for (rw::DBuf<double>* v : {&b->gx, &b->xx, &b->rx, &b->dx}) v->alloc(size_t(E) * nrhs);
    }
    if (b->dots.n < size_t(n) * nrhs) b->dots.alloc(size_t(n) * nrhs);
    ensure(b, nrhs);
    const size_t bytes = size_t(G) * nrhs * sizeof(double);
    const bool gdev = is_dev(g), tdev = is_dev(tau);
    RW_CUDA(cudaMemcpyAsync(b->gbuf.p, g, bytes, gdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    auto run = [&](const rw::Program& P, double* in, double* out) {
      double* bases[rw::kMaxBases] = {in, out, b->ws_ir.p, nullptr};
      P.run(bases, nrhs, s);
    };
    auto norms = [&](const double* a) {
      k_seg_dots<<<dim3(n, nrhs), 256, 0, s>>>(a, a, E, b->d_eoff.p, nrhs, b->dots.p);
      RW_CHECK_LAUNCH();
      std::vector<double> h(size_t(n) * nrhs);
      RW_CUDA(cudaMemcpyAsync(h.data(), b->dots.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      RW_CUDA(cudaStreamSynchronize(s));
      return h;
    };
    const size_t ne = size_t(E) * nrhs;
    run(b->p_in, b->gbuf.p, b->gx.p);
    run(b->p_dir, b->gx.p, b->xx.p);
    const std::vector<double> gn = norms(b->gx.p);
    for (;; ++it) {
      // r = g - (A~ + L R) x for every instance
      run(b->p_op, b->xx.p, b->rx.p);
      rw::axpby(b->gx.p, b->rx.p, ne, 1.0, -1.0, s);
      const std::vector<double> rn = norms(b->rx.p);
      worst = 0.0;
      for (size_t q = 0; q < rn.size(); ++q) worst = std::max(worst, gn[q] > 0 ? std::sqrt(rn[q] / gn[q]) : 0.0);
      if (worst <= tol || it >= maxit) break;
      run(b->p_dir, b->rx.p, b->dx.p);
      rw::axpby(b->dx.p, b->xx.p, ne, 1.0, 1.0, s);
    }
    run(b->p_out, b->xx.p, b->tbuf.p);
    RW_CUDA(cudaMemcpyAsync(tau, b->tbuf.p, bytes, tdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    RW_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres) *relres = worst;
    if (worst > tol)
      throw rw::Error(RW_ERR_NOT_CONVERGED,
                      "rw_batch_solve_ir: iterative refinement stopped at relative residual " + std::to_string(worst));
  } catch (const rw::Error& e) {
    if (iters) *iters = it;
    if (relres) *relres = worst;
    return rw::abi_fail(e.code, e.what());
  }
  rw::abi_clear_error();
  return RW_OK;
}

void rw_batch_free(rw_batch_t b) { delete b; }

}  // extern "C"
