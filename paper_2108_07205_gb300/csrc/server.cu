// Serving loop: continuous batching of refined-wall solve requests against
// resident reference walls.  A request is one local refinement of a wall
// (Algorithm 1's pre-computation) plus boundary data from point forces, the
// solve for nrhs right-hand sides and the velocity at targets.
//
// Requests wait in a FIFO queue and are admitted while the estimated device
// memory of the admitted requests and of the factor cache stays within the
// server's budget; each of n_workers host threads runs admitted requests end
// to end on its own CUDA stream (owned by the server), so the kernels of
// different requests overlap on the device.  When a request finishes, its
// memory is released (stream ordered) and waiting requests are admitted.
// Every request's result depends only on its own inputs (deterministic
// kernels and seeds), so it is the same alone and in the mix.
//
// Factor cache (optional, rw_server_set_cache): the pre-computation of a
// refinement is kept after its request, keyed by (wall, cut panels, levels),
// and a later request with the same key skips it (factor reuse across steps).
// Entries are evicted least recently used when the cache exceeds its
// capacity or when a waiting request needs the memory; solves on one cached
// refinement are serialised (they share its solve workspace).
#include "handles.cuh"
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <string>
#include <memory>
#include <mutex>
#include <thread>

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  long long ticket;
  const rw_hbs_s* wall;
  std::vector<int> panels, levels;
  int nrhs, n_src, n_targets, mode;
  std::vector<double> src, f, targets;
  double* tau;
  double* u;
  long long est_bytes;
  Clock::time_point t_submit, t_done;
  int status = 1;  // 1 pending/running, 0 ok, < 0 error
  std::string err;
};

}  // namespace

struct CachedRef {
  std::unique_ptr<rw::Refinement> ref;
  std::mutex solve_mu;  // one solve at a time on a cached refinement
  long long bytes = 0;
  int users = 0;
  unsigned long long last = 0;
};

struct rw_server_s {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<long long> queue;
  std::map<long long, Req> reqs;
  long long next_ticket = 1;
  long long budget = 0, in_use = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;  // one per worker; destroyed after the cache
  long long completed = 0;
  // factor cache
  long long cache_cap = 0, cache_bytes = 0, hits = 0, misses = 0;
  unsigned long long tick = 0;
  std::map<std::string, std::shared_ptr<CachedRef>> cache;

  void worker_loop(int w);
  // Moves the least recently used entry without users into `out`; false if
  // there is none.  mu held.
  bool evict_one(std::vector<std::shared_ptr<CachedRef>>& out) {
    auto best = cache.end();
    for (auto it = cache.begin(); it != cache.end(); ++it)
      if (it->second->users == 0 && (best == cache.end() || it->second->last < best->second->last)) best = it;
    if (best == cache.end()) return false;
    cache_bytes -= best->second->bytes;
    out.push_back(best->second);
    cache.erase(best);
    return true;
  }
};

namespace {

// Device bytes of one request (upper estimate): refined nodes and maps, the
// refined-arc HBS (~300 doubles per added unknown), the factors L, R, X at a
// Woodbury size of 512, the solve workspace and the ID scratch.
long long estimate_bytes(const rw_hbs_s* h, const std::vector<int>& levels, int nrhs) {
  const long long No = h->wall.nodes.n;
  long long Np = 0;
  for (int L : levels) Np += 16LL << L;
  const long long next2 = 2 * (No + Np);
  const long long k = 512;
  long long d = 0;
  d += next2 * k * 3;          // L, X (o and p parts), R
  d += 2 * Np * 300;           // A_pp HBS
  d += next2 * (8 + 6LL * nrhs);  // vectors, workspace
  d += 2 * No * 400;           // ID matrices (far rows x proxy features)
  return 8 * d + (64LL << 20);
}

std::string cache_key(const Req& r) {
  std::string k = std::to_string(reinterpret_cast<uintptr_t>(r.wall)) + "|";
  for (size_t i = 0; i < r.panels.size(); ++i) k += std::to_string(r.panels[i]) + ":" + std::to_string(r.levels[i]) + ",";
  return k;
}

}  // namespace

void rw_server_s::worker_loop(int wi) {
  const cudaStream_t s = streams[wi];
  rw::AllocStreamScope alloc_scope(s);  // every allocation of a request is stream ordered
  for (;;) {
    long long t = 0;
    Req* r = nullptr;
    std::vector<std::shared_ptr<CachedRef>> evicted;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (!queue.empty()) {
          const Req& head = reqs[queue.front()];
          // FIFO; cached factors give way to a waiting request; one request
          // always fits when nothing else runs
          while (in_use + cache_bytes + head.est_bytes > budget && evict_one(evicted)) {}
          if (in_use + cache_bytes + head.est_bytes <= budget || in_use == 0) break;
        } else if (stopping) {
          break;
        }
        cv_work.wait(lk);
      }
      if (queue.empty()) break;
      t = queue.front();
      queue.pop_front();
      r = &reqs[t];
      in_use += r->est_bytes;
    }
    evicted.clear();  // cached refinements freed outside the lock
    int status = RW_OK;
    std::string err;
    std::shared_ptr<CachedRef> ce;
    const std::string key = cache_key(*r);
    {
      std::lock_guard<std::mutex> lk(mu);
      if (cache_cap > 0) {
        auto it = cache.find(key);
        if (it != cache.end()) {
          ce = it->second;
          ++ce->users;
          ce->last = ++tick;
          ++hits;
        } else {
          ++misses;
        }
      }
    }
    std::unique_ptr<rw::Refinement> own;
    try {
      const rw::Refinement* refp = nullptr;
      if (ce) {
        refp = ce->ref.get();
      } else {
        own.reset(new rw::Refinement);
        own->factor(r->wall->wall, r->panels, r->levels, s);
        refp = own.get();
      }
      const rw::Refinement& ref = *refp;
      std::unique_lock<std::mutex> solve_lock;
      if (ce) solve_lock = std::unique_lock<std::mutex>(ce->solve_mu);
      const int Nn = ref.Nn;
      rw::TBuf<double> dsrc(r->src.size(), s), df(r->f.size(), s), dtg(std::max<size_t>(r->targets.size(), 1), s);
      RW_CUDA(cudaMemcpyAsync(dsrc.p, r->src.data(), r->src.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      RW_CUDA(cudaMemcpyAsync(df.p, r->f.data(), r->f.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      if (r->n_targets)
        RW_CUDA(cudaMemcpyAsync(dtg.p, r->targets.data(), r->targets.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      rw::TBuf<double> g(size_t(2) * Nn * r->nrhs, s), tau(size_t(2) * Nn * r->nrhs, s);
      rw::TBuf<double> u(size_t(2) * std::max(r->n_targets, 1) * r->nrhs, s);
      rw::eval_stokeslets(ref.nn.view(), r->n_src, dsrc.p, r->nrhs, df.p, g.p, s);
      int iters = 0;
      double relres = 0.0;
      const bool ir = r->mode == RW_MODE_DIRECT_IR || r->mode == RW_MODE_DIRECT_IR_DF;
      const bool gm = r->mode == RW_MODE_GMRES_FP32 || r->mode == RW_MODE_GMRES_BF16 ||
                      r->mode == RW_MODE_GMRES_MIXED || ir;
      if (ir) ref.solve_ir(g.p, tau.p, r->nrhs, s, &iters, &relres, r->mode == RW_MODE_DIRECT_IR_DF);
      else if (gm)
        ref.solve_gmres(g.p, tau.p, r->nrhs, s, &iters, &relres, r->mode == RW_MODE_GMRES_BF16,
                        r->mode == RW_MODE_GMRES_MIXED);
      else if (r->mode == RW_MODE_DIRECT_REFINED) ref.solve_refined(g.p, tau.p, r->nrhs, 1, s);
      else ref.solve_direct(g.p, tau.p, r->nrhs, s);
      if (r->n_targets) ref.velocity(tau.p, r->nrhs, r->n_targets, dtg.p, u.p, s);
      RW_CUDA(cudaMemcpyAsync(r->tau, tau.p, tau.n * sizeof(double), cudaMemcpyDeviceToHost, s));
      if (r->n_targets && r->u)
        RW_CUDA(cudaMemcpyAsync(r->u, u.p, size_t(2) * r->n_targets * r->nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
      RW_CUDA(cudaStreamSynchronize(s));
      if (gm && relres > r->wall->wall.opts.gmres_tol)
        throw rw::Error(RW_ERR_NOT_CONVERGED, "residual stopped at " + std::to_string(relres));
    } catch (const rw::Error& e) {
      status = e.code;
      err = e.what();
    } catch (const std::exception& e) {
      status = RW_ERR_INVALID;
      err = e.what();
    }
    cudaStreamSynchronize(s);
    {
      std::lock_guard<std::mutex> lk(mu);
      if (ce) --ce->users;
      // a new factorisation that fits joins the cache
      if (own && status == RW_OK && cache_cap > 0 && (long long)own->bytes <= cache_cap && !cache.count(key)) {
        auto e = std::make_shared<CachedRef>();
        e->bytes = (long long)own->bytes;
        e->ref = std::move(own);
        e->last = ++tick;
        cache_bytes += e->bytes;
        cache.emplace(key, e);
        while (cache_bytes > cache_cap && evict_one(evicted)) {}
      }
      r->status = status;
      r->err = err;
      r->t_done = Clock::now();
      in_use -= r->est_bytes;
      ++completed;
    }
    // the request's own refinement (if not cached) and evicted entries are
    // released here, stream ordered, outside the lock
    own.reset();
    evicted.clear();
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

namespace {
int sfail(int code, const std::string& m) { return rw::abi_fail(code, m); }
}  // namespace

extern "C" {

int rw_server_create(int n_workers, long long max_device_bytes, rw_server_t* out) {
  if (!out || n_workers < 1 || n_workers > 64 || max_device_bytes <= 0)
    return sfail(RW_ERR_INVALID, "rw_server_create: need 1..64 workers and a positive memory budget");
  rw_server_s* sv = new rw_server_s;
  sv->budget = max_device_bytes;
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < n_workers; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
      delete sv;
      return sfail(RW_ERR_CUDA, "rw_server_create: cannot create a worker stream");
    }
    sv->streams.push_back(st);
  }
  for (int i = 0; i < n_workers; ++i)
    sv->workers.emplace_back([sv, dev, i] {
      cudaSetDevice(dev);
      sv->worker_loop(i);
    });
  *out = sv;
  rw::abi_clear_error();
  return RW_OK;
}

int rw_server_set_cache(rw_server_t sv, long long max_bytes) {
  if (!sv || max_bytes < 0) return sfail(RW_ERR_INVALID, "rw_server_set_cache: bad argument");
  std::vector<std::shared_ptr<CachedRef>> evicted;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->cache_cap = max_bytes;
    while (sv->cache_bytes > sv->cache_cap && sv->evict_one(evicted)) {}
  }
  evicted.clear();
  sv->cv_work.notify_all();
  rw::abi_clear_error();
  return RW_OK;
}

int rw_server_stats(rw_server_t sv, long long* hits, long long* misses, long long* cache_bytes) {
  if (!sv) return sfail(RW_ERR_INVALID, "rw_server_stats: null server");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (hits) *hits = sv->hits;
  if (misses) *misses = sv->misses;
  if (cache_bytes) *cache_bytes = sv->cache_bytes;
  return RW_OK;
}

int rw_server_submit(rw_server_t sv, const rw_request* q, long long* ticket) {
  if (!sv || !q || !ticket || !q->wall || q->n_cut < 1 || !q->panel_ids || !q->levels || q->nrhs < 1 ||
      q->n_src < 1 || !q->src || !q->f || !q->tau || q->n_targets < 0 || (q->n_targets > 0 && (!q->targets || !q->u)))
    return sfail(RW_ERR_INVALID, "rw_server_submit: bad request");
  if (q->mode < RW_MODE_DIRECT || q->mode > RW_MODE_DIRECT_IR_DF)
    return sfail(RW_ERR_INVALID, "rw_server_submit: unknown mode");
  if (q->wall && q->wall->wall.opts.mixed_factor && (q->mode == RW_MODE_DIRECT || q->mode == RW_MODE_DIRECT_REFINED))
    return sfail(RW_ERR_INVALID, "rw_server_submit: walls with opts.mixed_factor take an iterative mode");
  Req r;
  r.wall = q->wall;
  r.panels.assign(q->panel_ids, q->panel_ids + q->n_cut);
  r.levels.assign(q->levels, q->levels + q->n_cut);
  for (int L : r.levels)
    if (L < 0 || L > 12) return sfail(RW_ERR_INVALID, "rw_server_submit: level must be in 0..12");
  r.nrhs = q->nrhs;
  r.n_src = q->n_src;
  r.n_targets = q->n_targets;
  r.mode = q->mode;
  r.src.assign(q->src, q->src + 2 * size_t(q->n_src));
  r.f.assign(q->f, q->f + 2 * size_t(q->n_src) * q->nrhs);
  if (q->n_targets) r.targets.assign(q->targets, q->targets + 2 * size_t(q->n_targets));
  r.tau = q->tau;
  r.u = q->u;
  r.est_bytes = estimate_bytes(q->wall, r.levels, q->nrhs);
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) return sfail(RW_ERR_INVALID, "rw_server_submit: server is stopping");
    r.ticket = sv->next_ticket++;
    *ticket = r.ticket;
    sv->reqs.emplace(r.ticket, std::move(r));
    sv->queue.push_back(*ticket);
  }
  sv->cv_work.notify_one();
  rw::abi_clear_error();
  return RW_OK;
}

int rw_server_poll(rw_server_t sv, long long ticket, int* status, double* latency_ms) {
  if (!sv || !status) return sfail(RW_ERR_INVALID, "rw_server_poll: bad argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return sfail(RW_ERR_INVALID, "rw_server_poll: unknown ticket");
  *status = it->second.status;
  if (latency_ms && it->second.status != 1)
    *latency_ms = std::chrono::duration<double, std::milli>(it->second.t_done - it->second.t_submit).count();
  return RW_OK;
}

int rw_server_wait(rw_server_t sv, long long ticket, double* latency_ms) {
  if (!sv) return sfail(RW_ERR_INVALID, "rw_server_wait: null server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return sfail(RW_ERR_INVALID, "rw_server_wait: unknown ticket");
  sv->cv_done.wait(lk, [&] { return it->second.status != 1; });
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(it->second.t_done - it->second.t_submit).count();
  const int st = it->second.status;
  if (st != RW_OK) {
    const std::string m = "request " + std::to_string(ticket) + ": " + it->second.err;
    lk.unlock();
    return sfail(st, m);
  }
  return RW_OK;
}

int rw_server_destroy(rw_server_t sv) {
  if (!sv) return RW_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->workers) t.join();
  // cached refinements release their memory on the worker streams, which go last
  sv->cache.clear();
  for (cudaStream_t st : sv->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  delete sv;
  return RW_OK;
}

}  // extern "C"
