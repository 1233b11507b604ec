// extern "C" boundary of the rwsolve library (declared in include/rwsolve.h).
// Argument checking, host/device pointer handling and error codes live here;
// the work is done by refine.cu / hbs.cu and the kernels below them.
#include "handles.cuh"
#include <cmath>
#include <cstring>
#include <memory>

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

template <class F>
int guarded(F&& f) {
  try {
    f();
    g_last_error.clear();
    return RW_OK;
  } catch (const rw::Error& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(RW_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(RW_ERR_INVALID, e.what());
  }
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller buffer: the pointer itself if it is device memory,
// else a stream-ordered copy (copied in if `in`, copied back by `finish`).
struct Arg {
  const void* user = nullptr;
  size_t bytes = 0;
  bool device = true;
  rw::TBuf<double> tmp;
  double* p = nullptr;
  Arg(const double* u, size_t count, bool in, cudaStream_t s) : user(u), bytes(count * sizeof(double)) {
    if (!u || !count) { p = const_cast<double*>(u); return; }
    device = is_device_ptr(u);
    if (device) { p = const_cast<double*>(u); return; }
    tmp = rw::TBuf<double>(count, s);
    p = tmp.p;
    if (in) RW_CUDA(cudaMemcpyAsync(p, u, bytes, cudaMemcpyHostToDevice, s));
  }
  void finish(cudaStream_t s) {
    if (!device && bytes) {
      RW_CUDA(cudaMemcpyAsync(const_cast<void*>(user), p, bytes, cudaMemcpyDeviceToHost, s));
    }
  }
};

rw::Opts to_opts(const rw_opts* o) {
  rw::Opts r;
  if (!o) return r;
  rw::require(o->leaf_points >= 8 && o->leaf_points <= 512, "opts.leaf_points must be in 8..512");
  rw::require(o->id_tol > 0 && o->id_tol < 1, "opts.id_tol must be in (0, 1)");
  rw::require(o->n_proxy >= 8 && o->n_proxy <= 1024, "opts.n_proxy must be in 8..1024");
  rw::require(o->proxy_ratio > 1.0, "opts.proxy_ratio must exceed 1");
  rw::require(o->n_proxy_refine >= 8 && o->n_proxy_refine <= 1024, "opts.n_proxy_refine must be in 8..1024");
  rw::require(o->div_ratio > o->bas_ratio && o->bas_ratio > 1.0, "opts need div_ratio > bas_ratio > 1");
  rw::require(o->hole_div_ratio > o->bas_ratio, "opts need hole_div_ratio > bas_ratio");
  rw::require(o->sketch_cols >= 64, "opts.sketch_cols must be >= 64");
  rw::require(o->gmres_tol > 0 && o->gmres_maxit >= 1 && o->gmres_restarts >= 1, "bad GMRES options");
  rw::require(o->op_tol == 0.0 || (o->op_tol > 0 && o->op_tol < 1), "opts.op_tol must be 0 or in (0, 1)");
  rw::require(o->mixed_factor >= 0 && o->mixed_factor <= 2, "opts.mixed_factor must be 0, 1 or 2");
  r.leaf_points = o->leaf_points;
  r.id_tol = o->id_tol;
  r.n_proxy = o->n_proxy;
  r.proxy_ratio = o->proxy_ratio;
  r.n_proxy_refine = o->n_proxy_refine;
  r.div_ratio = o->div_ratio;
  r.bas_ratio = o->bas_ratio;
  r.dense_pp_max_points = o->dense_pp_max_points;
  r.sketch_cols = o->sketch_cols;
  r.gmres_tol = o->gmres_tol;
  r.gmres_maxit = o->gmres_maxit;
  r.gmres_restarts = o->gmres_restarts;
  r.seed = o->seed;
  r.hole_div_ratio = o->hole_div_ratio;
  r.op_tol = o->op_tol;
  r.mixed_factor = o->mixed_factor;
  return r;
}

// Copies the six arrays of an rw_nodes (host or device) into one host
// array, 6 x n column-major (x, y, nx, ny, w, kappa), and checks them.
std::vector<double> stage_nodes(const rw_nodes* nd, int n_expected, const char* what, cudaStream_t s) {
  rw::require(nd != nullptr, std::string(what) + ": null nodes");
  const int n = nd->n;
  rw::require(n >= 16 && n % 16 == 0, std::string(what) + ": n must be a positive multiple of 16");
  rw::require(n_expected < 0 || n == n_expected,
              std::string(what) + ": expected " + std::to_string(n_expected) + " nodes, got " + std::to_string(n));
  const double* src[6] = {nd->x, nd->y, nd->nx, nd->ny, nd->w, nd->kappa};
  std::vector<double> h(6 * size_t(n));
  for (int c = 0; c < 6; ++c) {
    rw::require(src[c] != nullptr, std::string(what) + ": null node array");
    RW_CUDA(cudaMemcpyAsync(h.data() + size_t(c) * n, src[c], size_t(n) * sizeof(double), cudaMemcpyDefault, s));
  }
  RW_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i) {
    for (int c = 0; c < 6; ++c)
      rw::require(std::isfinite(h[size_t(c) * n + i]), std::string(what) + ": non-finite node data");
    const double nx = h[2 * size_t(n) + i], ny = h[3 * size_t(n) + i];
    rw::require(std::fabs(nx * nx + ny * ny - 1.0) <= 1e-8, std::string(what) + ": normals must have unit length");
    rw::require(h[4 * size_t(n) + i] > 0.0, std::string(what) + ": weights must be positive");
  }
  return h;
}

}  // namespace

namespace rw {
int abi_fail(int code, const std::string& msg) { return fail(code, msg); }
void abi_clear_error() { g_last_error.clear(); }
}  // namespace rw

extern "C" {

int rw_default_opts(rw_opts* o) {
  if (!o) return fail(RW_ERR_INVALID, "rw_default_opts: null");
  rw::Opts d;
  o->leaf_points = d.leaf_points;
  o->id_tol = d.id_tol;
  o->n_proxy = d.n_proxy;
  o->proxy_ratio = d.proxy_ratio;
  o->n_proxy_refine = d.n_proxy_refine;
  o->div_ratio = d.div_ratio;
  o->bas_ratio = d.bas_ratio;
  o->dense_pp_max_points = d.dense_pp_max_points;
  o->sketch_cols = d.sketch_cols;
  o->gmres_tol = d.gmres_tol;
  o->gmres_maxit = d.gmres_maxit;
  o->gmres_restarts = d.gmres_restarts;
  o->seed = d.seed;
  o->hole_div_ratio = d.hole_div_ratio;
  o->op_tol = d.op_tol;
  o->mixed_factor = d.mixed_factor;
  return RW_OK;
}

namespace {
int build_curve_wall(const rw_wall_desc* wd, const rw_opts* opts, void* stream, rw_hbs_t* out, bool exterior);
}  // namespace

int rw_hbs_build(const rw_wall_desc* wd, const rw_opts* opts, void* stream, rw_hbs_t* out) {
  return build_curve_wall(wd, opts, stream, out, false);
}

int rw_hbs_build_exterior(const rw_wall_desc* wd, const rw_opts* opts, void* stream, rw_hbs_t* out) {
  return build_curve_wall(wd, opts, stream, out, true);
}

namespace {
int build_curve_wall(const rw_wall_desc* wd, const rw_opts* opts, void* stream, rw_hbs_t* out, bool exterior) {
  if (!wd || !out) return fail(RW_ERR_INVALID, exterior ? "rw_hbs_build_exterior: null argument"
                                                         : "rw_hbs_build: null argument");
  *out = nullptr;
  std::unique_ptr<rw_hbs_s> h(new rw_hbs_s);
  int rc = guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rw::Wall& w = h->wall;
    w.opts = to_opts(opts);
    rw::require(wd->n_panels >= 1 && wd->n_panels <= (1 << 20), "wall.n_panels must be in 1..2^20");
    rw::require(!exterior || wd->n_panels >= 8, "exterior wall: at least 8 panels");
    w.n_panels = wd->n_panels;
    w.curve.kind = wd->curve_kind;
    for (int i = 0; i < 8; ++i) w.curve.p[i] = wd->params[i];
    if (wd->curve_kind == RW_CURVE_STAR) {
      if (w.curve.p[2] == 0.0) w.curve.p[2] = 1.0;
      rw::require(std::fabs(w.curve.p[0]) < 1.0 && w.curve.p[2] > 0, "star: need |a| < 1 and scale > 0");
    } else if (wd->curve_kind == RW_CURVE_CHANNEL) {
      const double def[4] = {10.0, 0.5, 8.0, 0.6};
      bool all0 = true;
      for (int i = 0; i < 4; ++i) all0 = all0 && w.curve.p[i] == 0.0;
      if (all0) for (int i = 0; i < 4; ++i) w.curve.p[i] = def[i];
      rw::require(w.curve.p[0] > 0 && w.curve.p[1] > 0 && w.curve.p[2] >= 2 && w.curve.p[3] >= 0 && w.curve.p[3] < 1,
                  "channel: need A > 0, B > 0, p >= 2 (even), 0 <= delta < 1");
    } else {
      throw rw::Error(RW_ERR_INVALID, "unknown curve kind");
    }
    const int P = w.n_panels;
    std::vector<double> ta(P), tb(P);
    for (int j = 0; j < P; ++j) { ta[j] = 2.0 * rw::kPi * j / P; tb[j] = 2.0 * rw::kPi * (j + 1) / P; }
    auto dta = rw::to_device_tmp(ta, s), dtb = rw::to_device_tmp(tb, s);
    w.nodes.alloc(16 * P);
    rw::eval_nodes(w.curve, dta.p, dtb.p, P, w.nodes.buf.p, 16 * P, s);
    auto all = w.nodes.buf.download(s);
    w.nodes.hx.assign(all.begin(), all.begin() + 16 * P);
    w.nodes.hy.assign(all.begin() + 16 * P, all.begin() + 32 * P);
    if (exterior) rw::set_exterior_panels(w.nodes, w.curve, ta, tb, s);
    w.build_hbs(s);
  });
  if (rc == RW_OK) *out = h.release();
  return rc;
}
}  // namespace

int rw_hbs_build_nodes(const rw_nodes* nodes, const rw_opts* opts, void* stream, rw_hbs_t* out) {
  if (!nodes || !out) return fail(RW_ERR_INVALID, "rw_hbs_build_nodes: null argument");
  *out = nullptr;
  std::unique_ptr<rw_hbs_s> h(new rw_hbs_s);
  int rc = guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rw::Wall& w = h->wall;
    w.opts = to_opts(opts);
    const std::vector<double> hn = stage_nodes(nodes, -1, "rw_hbs_build_nodes", s);
    const int n = nodes->n;
    rw::require(n / 16 <= (1 << 20), "rw_hbs_build_nodes: at most 2^20 panels");
    w.n_panels = n / 16;
    w.curve.kind = RW_CURVE_NODES;
    for (int i = 0; i < 8; ++i) w.curve.p[i] = 0.0;
    w.nodes.alloc(n);
    RW_CUDA(cudaMemcpyAsync(w.nodes.buf.p, hn.data(), hn.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    w.nodes.hx.assign(hn.begin(), hn.begin() + n);
    w.nodes.hy.assign(hn.begin() + n, hn.begin() + 2 * size_t(n));
    w.build_hbs(s);
  });
  if (rc == RW_OK) *out = h.release();
  return rc;
}

int rw_hbs_stats_get(rw_hbs_t h, rw_hbs_stats* st) {
  if (!h || !st) return fail(RW_ERR_INVALID, "rw_hbs_stats_get: null argument");
  const rw::Hbs& b = h->wall.hbs;
  st->n_points = b.N;
  st->levels = b.L;
  st->max_rank = b.max_rank;
  st->inv_elems = b.inv_elems;
  st->fwd_elems = b.fwd_elems;
  st->bytes = (long long)(b.bytes + h->wall.hbs_op.bytes + h->wall.nodes.buf.bytes());
  st->op_fwd_elems = h->wall.op().fwd_elems;
  return RW_OK;
}

int rw_hbs_nodes(rw_hbs_t h, double* out, void* stream) {
  if (!h || !out) return fail(RW_ERR_INVALID, "rw_hbs_nodes: null argument");
  return guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const auto& b = h->wall.nodes.buf;
    RW_CUDA(cudaMemcpyAsync(out, b.p, b.bytes(), cudaMemcpyDefault, s));
    RW_CUDA(cudaStreamSynchronize(s));
  });
}

int rw_hbs_apply_inverse(rw_hbs_t h, int nrhs, const double* b, double* x, void* stream) {
  if (!h || !b || !x || nrhs < 1) return fail(RW_ERR_INVALID, "rw_hbs_apply_inverse: bad argument");
  if (b == x) return fail(RW_ERR_INVALID, "rw_hbs_apply_inverse: b and x may not alias");
  return guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = size_t(2) * h->wall.nodes.n * nrhs;
    Arg ab(b, n, true, s), ax(x, n, false, s);
    h->wall.hbs.apply_inverse(ab.p, ax.p, nrhs, s);
    ax.finish(s);
    RW_CUDA(cudaStreamSynchronize(s));
  });
}

int rw_hbs_apply_forward(rw_hbs_t h, int nrhs, const double* x, double* y, void* stream) {
  if (!h || !x || !y || nrhs < 1) return fail(RW_ERR_INVALID, "rw_hbs_apply_forward: bad argument");
  if (x == y) return fail(RW_ERR_INVALID, "rw_hbs_apply_forward: x and y may not alias");
  return guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = size_t(2) * h->wall.nodes.n * nrhs;
    Arg ax(x, n, true, s), ay(y, n, false, s);
    h->wall.hbs.apply_forward(ax.p, ay.p, nrhs, s);
    ay.finish(s);
    RW_CUDA(cudaStreamSynchronize(s));
  });
}

int rw_refine_factor(rw_hbs_t h, int n_cut, const int* panel_ids, const int* levels, void* stream, rw_ref_t* out) {
  if (!h || !panel_ids || !levels || !out || n_cut < 1) return fail(RW_ERR_INVALID, "rw_refine_factor: bad argument");
  *out = nullptr;
  std::unique_ptr<rw_ref_s> r(new rw_ref_s);
  r->h = h;
  int rc = guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rw::require(h->wall.curve.kind != RW_CURVE_NODES,
                "rw_refine_factor: this wall was built from nodes; give the added nodes (rw_refine_factor_nodes)");
    std::vector<int> pan(panel_ids, panel_ids + n_cut), lv(levels, levels + n_cut);
    r->ref.factor(h->wall, pan, lv, s);
    RW_CUDA(cudaStreamSynchronize(s));
  });
  if (rc == RW_OK) *out = r.release();
  return rc;
}

int rw_refine_factor_nodes(rw_hbs_t h, int n_cut, const int* panel_ids, const int* levels, const rw_nodes* added,
                           void* stream, rw_ref_t* out) {
  if (!h || !panel_ids || !levels || !added || !out || n_cut < 1)
    return fail(RW_ERR_INVALID, "rw_refine_factor_nodes: bad argument");
  *out = nullptr;
  std::unique_ptr<rw_ref_s> r(new rw_ref_s);
  r->h = h;
  int rc = guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int> pan(panel_ids, panel_ids + n_cut), lv(levels, levels + n_cut);
    long long np = 0;
    for (int L : lv) {
      rw::require(L >= 0 && L <= 12, "rw_refine_factor_nodes: level must be in 0..12");
      np += 16LL << L;
    }
    rw::require(np <= (1LL << 30), "rw_refine_factor_nodes: too many added nodes");
    const std::vector<double> hn = stage_nodes(added, int(np), "rw_refine_factor_nodes", s);
    r->ref.factor(h->wall, pan, lv, s, &hn);
    RW_CUDA(cudaStreamSynchronize(s));
  });
  if (rc == RW_OK) *out = r.release();
  return rc;
}

int rw_holes_factor(rw_hbs_t h, int n_holes, const rw_hole* holes, void* stream, rw_ref_t* out) {
  if (!h || !holes || !out || n_holes < 1) return fail(RW_ERR_INVALID, "rw_holes_factor: bad argument");
  *out = nullptr;
  std::unique_ptr<rw_ref_s> r(new rw_ref_s);
  r->h = h;
  int rc = guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<rw::HoleSpec> hs;
    for (int i = 0; i < n_holes; ++i)
      hs.push_back(rw::HoleSpec{holes[i].cx, holes[i].cy, holes[i].radius, holes[i].a, holes[i].k, holes[i].n_panels});
    r->ref.factor_holes(h->wall, hs, s);
    RW_CUDA(cudaStreamSynchronize(s));
  });
  if (rc == RW_OK) *out = r.release();
  return rc;
}

int rw_ref_stats_get(rw_ref_t r, rw_ref_stats* st) {
  if (!r || !st) return fail(RW_ERR_INVALID, "rw_ref_stats_get: null argument");
  const rw::Refinement& f = r->ref;
  st->n_k = f.Nk; st->n_c = f.Nc; st->n_p = f.Np; st->n_n = f.Nn; st->n_ext = f.Nk + f.Nc + f.Np;
  st->k_far = f.kf; st->k_near = f.kn; st->k_pk = f.kpk_id; st->k = f.k;
  st->pp_dense = f.pp_dense ? 1 : 0;
  st->pp_levels = f.pp_dense ? 0 : f.hpp.L;
  st->bytes = (long long)f.bytes;
  return RW_OK;
}

int rw_ref_nodes(rw_ref_t r, double* out, void* stream) {
  if (!r || !out) return fail(RW_ERR_INVALID, "rw_ref_nodes: null argument");
  return guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const auto& b = r->ref.nn.buf;
    RW_CUDA(cudaMemcpyAsync(out, b.p, b.bytes(), cudaMemcpyDefault, s));
    RW_CUDA(cudaStreamSynchronize(s));
  });
}

int rw_apply_refined(rw_ref_t r, int nrhs, const double* tau, double* y, void* stream) {
  if (!r || !tau || !y || nrhs < 1) return fail(RW_ERR_INVALID, "rw_apply_refined: bad argument");
  if (tau == y) return fail(RW_ERR_INVALID, "rw_apply_refined: tau and y may not alias");
  return guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = size_t(2) * r->ref.Nn * nrhs;
    Arg at(tau, n, true, s), ay(y, n, false, s);
    r->ref.apply_nn(at.p, ay.p, nrhs, s);
    ay.finish(s);
    RW_CUDA(cudaStreamSynchronize(s));
  });
}

int rw_stokeslet_data(rw_ref_t r, int n_src, const double* src, int nrhs, const double* f, double* g, void* stream) {
  if (!r || !src || !f || !g || n_src < 1 || nrhs < 1) return fail(RW_ERR_INVALID, "rw_stokeslet_data: bad argument");
  return guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Arg as(src, size_t(2) * n_src, true, s), af(f, size_t(2) * n_src * nrhs, true, s);
    Arg ag(g, size_t(2) * r->ref.Nn * nrhs, false, s);
    rw::eval_stokeslets(r->ref.nn.view(), n_src, as.p, nrhs, af.p, ag.p, s);
    ag.finish(s);
    RW_CUDA(cudaStreamSynchronize(s));
  });
}

int rw_solve(rw_ref_t r, int nrhs, const double* g, double* tau, int n_targets, const double* targets, double* u,
             int mode, void* stream, rw_info* info) {
  if (!r || !g || !tau || nrhs < 1 || n_targets < 0) return fail(RW_ERR_INVALID, "rw_solve: bad argument");
  if (n_targets > 0 && (!targets || !u)) return fail(RW_ERR_INVALID, "rw_solve: targets and u required");
  if (mode < RW_MODE_DIRECT || mode > RW_MODE_DIRECT_IR_DF) return fail(RW_ERR_INVALID, "rw_solve: unknown mode");
  if (r->ref.wall->opts.mixed_factor && (mode == RW_MODE_DIRECT || mode == RW_MODE_DIRECT_REFINED))
    return fail(RW_ERR_INVALID,
                "rw_solve: this refinement's X is not FP64 (opts.mixed_factor): use an iterative mode");
  int iters = 0;
  double relres = 0.0;
  int rc = guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const rw::Refinement& f = r->ref;
    const size_t n = size_t(2) * f.Nn * nrhs;
    Arg ag(g, n, true, s), at(tau, n, false, s);
    if (mode == RW_MODE_DIRECT) {
      f.solve_direct(ag.p, at.p, nrhs, s);
    } else if (mode == RW_MODE_DIRECT_REFINED) {
      f.solve_refined(ag.p, at.p, nrhs, 1, s);
      iters = 1;
    } else if (mode == RW_MODE_DIRECT_IR || mode == RW_MODE_DIRECT_IR_DF) {
      f.solve_ir(ag.p, at.p, nrhs, s, &iters, &relres, mode == RW_MODE_DIRECT_IR_DF);
    } else {
      f.solve_gmres(ag.p, at.p, nrhs, s, &iters, &relres, mode == RW_MODE_GMRES_BF16, mode == RW_MODE_GMRES_MIXED);
    }
    if (n_targets > 0) {
      Arg ax(targets, size_t(2) * n_targets, true, s), au(u, size_t(2) * n_targets * nrhs, false, s);
      f.velocity(at.p, nrhs, n_targets, ax.p, au.p, s);
      au.finish(s);
    }
    at.finish(s);
    RW_CUDA(cudaStreamSynchronize(s));
    if ((mode == RW_MODE_GMRES_FP32 || mode == RW_MODE_GMRES_BF16 || mode == RW_MODE_GMRES_MIXED) &&
        relres > f.wall->opts.gmres_tol)
      throw rw::Error(RW_ERR_NOT_CONVERGED, "rw_solve: GMRES stopped at relative residual " + std::to_string(relres));
    if ((mode == RW_MODE_DIRECT_IR || mode == RW_MODE_DIRECT_IR_DF) && relres > f.wall->opts.gmres_tol)
      throw rw::Error(RW_ERR_NOT_CONVERGED,
                      "rw_solve: iterative refinement stopped at relative residual " + std::to_string(relres));
  });
  if (info) {
    info->iters = iters;
    info->rel_residual = relres;
    info->k_woodbury = r->ref.k;
    info->cond_w = r->ref.cond_w;
  }
  return rc;
}

int rw_pressure(rw_ref_t r, int nrhs, const double* tau, int n_targets, const double* targets, double* p,
                void* stream) {
  if (!r || !tau || !targets || !p || nrhs < 1 || n_targets < 1) return fail(RW_ERR_INVALID, "rw_pressure: bad argument");
  return guarded([&] {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const rw::Refinement& f = r->ref;
    Arg at(tau, size_t(2) * f.Nn * nrhs, true, s), ax(targets, size_t(2) * n_targets, true, s);
    Arg ap(p, size_t(n_targets) * nrhs, false, s);
    f.pressure(at.p, nrhs, n_targets, ax.p, ap.p, s);
    ap.finish(s);
    RW_CUDA(cudaStreamSynchronize(s));
  });
}

unsigned long long rw_kernel_launches(void) { return rw::g_launches; }

int rw_profile(int enable) {
  return guarded([&] { rw::profile_enable(enable != 0); });
}

int rw_profile_read(rw_kernel_stat* out, int n) {
  if (!out || n < RW_KCLASS_COUNT) return fail(RW_ERR_INVALID, "rw_profile_read: need RW_KCLASS_COUNT entries");
  return guarded([&] {
    long long l[rw::KC_COUNT];
    double ms[rw::KC_COUNT], fl[rw::KC_COUNT], by[rw::KC_COUNT];
    rw::profile_read(l, ms, fl, by);
    for (int c = 0; c < RW_KCLASS_COUNT; ++c) {
      out[c].launches = l[c];
      out[c].ms = ms[c];
      out[c].flops = fl[c];
      out[c].bytes = by[c];
    }
  });
}

void rw_ref_free(rw_ref_t r) { delete r; }
void rw_hbs_free(rw_hbs_t h) { delete h; }
const char* rw_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
