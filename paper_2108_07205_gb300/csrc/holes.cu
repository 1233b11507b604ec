// Algorithm 1 for the wall with added holes (App. B, Eq. simple_ext): no
// point is cut, the holes' points are the added set I_p, and the update of
// blkdiag(A_kk, A_pp) is Q = [0 A_kp; A_pk 0].
//
// Low-rank factors (Sec. 3.3 with one proxy circle per hole, as the paper
// does for its three holes):
//  * wall rows outside every hole's P^div circle: one hierarchical ID of
//    A_kp against proxy sources on the union of the holes' P^bas circles;
//  * wall rows inside some P^div circle: one direct ID of A_kp^near;
//  * A_pk, hole by hole: a hierarchical ID of the hole's rows of
//    [A_{p,div} | A_pk^near] with that hole's P^div circle and the wall
//    points inside it; L_pk = blkdiag over the holes.
// so L = blkdiag(L_k, L_pk), R = [[0, A(J_k, I_p)], [A(J_pk, I_k), 0]],
// with the wall block recompressed by a row ID of its skeleton rows
// (Sec. 3.4).
// A_pp = 1/2 I + D + S is assembled densely with the singular rule of the
// hole matrix kernel and inverted (single-leaf HBS).
#include "refine.cuh"
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <exception>
#include <thread>

namespace rw {

void Refinement::factor_holes(const Wall& w, const std::vector<HoleSpec>& hs, cudaStream_t s) {
  require(w.nodes.kind != kNodesExterior, "holes: the wall must enclose the fluid (an interior wall)");
  wall = &w;
  holes = true;
  streams.main = s;
  AllocStreamScope alloc_scope(s);
  Trace tr(s, "holes");
  const Opts& o = w.opts;
  // IDs (and A_pp) at the operator tolerance when that is tighter: the
  // factors then serve as the accurate operator for residuals as well
  const double ftol = o.factor_tol();
  const int nh = int(hs.size());
  require(nh >= 1 && nh <= 8, "holes: 1 to 8 holes");
  int np = 0;
  for (const HoleSpec& h : hs) {
    require(std::isfinite(h.cx) && std::isfinite(h.cy) && std::isfinite(h.R) && std::isfinite(h.a),
            "holes: non-finite hole parameter");
    require(h.R > 0.0, "holes: radius must be positive");
    require(h.a >= 0.0 && h.a < 1.0, "holes: shape amplitude a must be in [0, 1)");
    require(h.k >= 0 && h.k <= 64, "holes: shape frequency k must be in 0..64");
    require(h.P >= 5 && h.P <= 256, "holes: 5 to 256 panels per hole");
    np += 16 * h.P;
  }
  require(np <= 1024, "holes: at most 1024 hole points (A_pp is inverted densely)");
  for (int a = 0; a < nh; ++a)
    for (int b = a + 1; b < nh; ++b) {
      const double d = std::hypot(hs[a].cx - hs[b].cx, hs[a].cy - hs[b].cy);
      require(d > hs[a].R * (1.0 + hs[a].a) + hs[b].R * (1.0 + hs[b].a), "holes: holes overlap");
    }
  panels.clear();
  levels.clear();
  No = w.nodes.n;
  Nc = 0;
  Nk = No;
  Np = np;
  Nn = No + Np;
  Ic.clear();
  Ik.resize(No);
  for (int i = 0; i < No; ++i) Ik[i] = i;

  // a1: hole nodes (hole by hole, panels equal in t)
  pn.alloc(Np);
  pn.kind = 1;
  {
    std::vector<double> ta, tb;
    for (const HoleSpec& h : hs)
      for (int j = 0; j < h.P; ++j) {
        ta.push_back(2.0 * kPi * j / h.P);
        tb.push_back(2.0 * kPi * (j + 1) / h.P);
      }
    auto dta = to_device_tmp(ta, s), dtb = to_device_tmp(tb, s);
    int off = 0, poff = 0;
    for (const HoleSpec& h : hs) {
      Curve c{kCurveHole, {h.a, double(h.k), h.R, h.cx, h.cy, 0.0, 0.0, 0.0}};
      eval_nodes(c, dta.p + poff, dtb.p + poff, h.P, pn.buf.p + off, Np, s);
      off += 16 * h.P;
      poff += h.P;
    }
    auto all = pn.buf.download(s);
    pn.hx.assign(all.begin(), all.begin() + Np);
    pn.hy.assign(all.begin() + Np, all.begin() + 2 * Np);
  }
  // refined order: the wall's points, then the holes' points
  {
    std::vector<int> from_o(2 * No), from_p(2 * Np), to_p(2 * Np);
    for (int d = 0; d < 2 * No; ++d) from_o[d] = d;
    for (int d = 0; d < 2 * Np; ++d) { from_p[d] = 2 * No + d; to_p[d] = d; }
    n_from_o = to_device(from_o, s);
    n_to_o = to_device(from_o, s);
    n_from_p = to_device(from_p, s);
    n_to_p = to_device(to_p, s);
    nko = 2 * No;
    nkp = 2 * Np;
    nn.alloc(Nn);
    for (int c = 0; c < 6; ++c) {
      RW_CUDA(cudaMemcpyAsync(nn.buf.p + size_t(c) * Nn, w.nodes.buf.p + size_t(c) * No, sizeof(double) * No,
                              cudaMemcpyDeviceToDevice, s));
      RW_CUDA(cudaMemcpyAsync(nn.buf.p + size_t(c) * Nn + No, pn.buf.p + size_t(c) * Np, sizeof(double) * Np,
                              cudaMemcpyDeviceToDevice, s));
    }
    RW_CUDA(cudaStreamSynchronize(s));
  }
  tr.mark("nodes+maps");
  // per hole: centre and radius of its points, P^div and P^bas circles
  std::vector<double> hcx(nh), hcy(nh), hrho(nh), circ_bas, circ_div;
  std::vector<int> hoff(nh + 1, 0);
  for (int h = 0; h < nh; ++h) hoff[h + 1] = hoff[h] + 16 * hs[h].P;
  for (int h = 0; h < nh; ++h) {
    double cx = 0, cy = 0, r2 = 0;
    for (int i = hoff[h]; i < hoff[h + 1]; ++i) { cx += pn.hx[i]; cy += pn.hy[i]; }
    cx /= (hoff[h + 1] - hoff[h]);
    cy /= (hoff[h + 1] - hoff[h]);
    for (int i = hoff[h]; i < hoff[h + 1]; ++i)
      r2 = std::max(r2, (pn.hx[i] - cx) * (pn.hx[i] - cx) + (pn.hy[i] - cy) * (pn.hy[i] - cy));
    hcx[h] = cx;
    hcy[h] = cy;
    hrho[h] = std::sqrt(r2);
    circ_bas.insert(circ_bas.end(), {cx, cy, o.bas_ratio * hrho[h]});
    circ_div.insert(circ_div.end(), {cx, cy, o.hole_div_ratio * hrho[h]});
  }
  // wall DOFs: far (outside every P^div circle) and near; near set per hole
  std::vector<int> far_d, near_d;
  std::vector<std::vector<int>> near_h(nh);
  for (int i = 0; i < No; ++i) {
    bool near = false;
    for (int h = 0; h < nh; ++h) {
      const double dx = w.nodes.hx[i] - hcx[h], dy = w.nodes.hy[i] - hcy[h];
      if (dx * dx + dy * dy < circ_div[3 * h + 2] * circ_div[3 * h + 2]) {
        near = true;
        near_h[h].push_back(2 * i);
        near_h[h].push_back(2 * i + 1);
      }
    }
    auto& v = near ? near_d : far_d;
    v.push_back(2 * i);
    v.push_back(2 * i + 1);
  }

  const NodesView VW = w.nodes.view(), VP = pn.view();
  TreeId tf, tn;
  std::vector<TreeId> tp(nh);
  DBuf<int> dall_p = [&] {
    std::vector<int> pd(2 * Np);
    for (int i = 0; i < 2 * Np; ++i) pd[i] = i;
    return to_device(pd, s);
  }();
  DBuf<double> dcirc_bas = to_device(circ_bas, s);
  std::vector<DBuf<int>> dnear_h(nh);
  for (int h = 0; h < nh; ++h) dnear_h[h] = to_device(near_h[h], s);
  RW_CUDA(cudaStreamSynchronize(s));
  RW_CUDA(cudaStreamCreateWithFlags(&streams.s1, cudaStreamNonBlocking));
  RW_CUDA(cudaStreamCreateWithFlags(&streams.s2, cudaStreamNonBlocking));
  cudaStream_t s1 = streams.s1, s2 = streams.s2;
  std::exception_ptr e1, e2, e0;
  // a2 (A_pp, dense with the singular rule, and its inverse) and the far ID
  // run on their own streams while the near and A_pk IDs run on the main one
  auto task1 = [&] {
    AllocStreamScope scope1(s1);
    try {
      DBuf<double> A(size_t(4) * Np * Np);
      std::vector<int> pan(nh);
      std::vector<double> geo;
      for (int h = 0; h < nh; ++h) {
        pan[h] = hs[h].P;
        geo.insert(geo.end(), {hs[h].a, double(hs[h].k), hs[h].R, hs[h].cx, hs[h].cy});
      }
      eval_hole_matrix(VP, pan, geo, A.p, s1);
      hpp.build_dense(std::move(A), Np, s1);
      hpp.own_stream = s;   // later copies and programs live on the refinement's stream
      hpp.make_fp32(s1);
      hpp.make_bf16(s1);
      pp_dense = true;
      RW_CUDA(cudaStreamSynchronize(s1));
    } catch (...) { e1 = std::current_exception(); }
  };
  auto task2 = [&] {
    AllocStreamScope scope2(s2);
    try {
      IdMatProb cs{};
      cs.M = o.n_proxy_refine;
      cs.normal = 0;
      cs.ncirc = nh;
      cs.circ = dcirc_bas.p;
      if (nh == 1) { cs.cx = circ_bas[0]; cs.cy = circ_bas[1]; cs.R = circ_bas[2]; cs.ncirc = 0; cs.circ = nullptr; }
      tf = tree_row_id(VW, far_d, cs, VW, true, VW, true, ftol, o.sketch_cols, o.sketch_width, o.seed + 101, 128, s2);
    } catch (...) { e2 = std::current_exception(); }
  };
  std::thread th1(task1), th2(task2);
  struct Joiner {
    std::thread& t;
    ~Joiner() { if (t.joinable()) t.join(); }
  } join1{th1}, join2{th2};
  try {
    // near wall rows: [A_kp^near] against every hole DOF
    {
      IdMatProb cs{};
      cs.n2 = 2 * Np; cs.e2 = dall_p.p; cs.M = 0; cs.normal = 0;
      tn = tree_row_id(VW, near_d, cs, VW, true, VP, false, ftol, o.sketch_cols, o.sketch_width, o.seed + 202, 128, s);
    }
    // A_pk per hole: rows of [A_{p,div} | A_pk^near]
    for (int h = 0; h < nh; ++h) {
      std::vector<int> prow;
      for (int d = 2 * hoff[h]; d < 2 * hoff[h + 1]; ++d) prow.push_back(d);
      IdMatProb cs{};
      cs.n1 = int(near_h[h].size()); cs.e1 = dnear_h[h].p;
      cs.cx = circ_div[3 * h]; cs.cy = circ_div[3 * h + 1]; cs.R = circ_div[3 * h + 2];
      cs.M = o.n_proxy_refine; cs.normal = 0;
      tp[h] = tree_row_id(VP, prow, cs, VW, false, VW, false, ftol, o.sketch_cols, o.sketch_width,
                          o.seed + 303 + h, 128, s);
    }
  } catch (...) { e0 = std::current_exception(); }
  if (th2.joinable()) th2.join();
  RW_CUDA(cudaStreamSynchronize(s2));
  for (auto& e : {e0, e2}) if (e) std::rethrow_exception(e);
  tr.mark("IDs (concurrent with A_pp)");
  kf = tf.k;
  kn = tn.k;
  kpk = 0;
  for (int h = 0; h < nh; ++h) kpk += tp[h].k;
  kk = kf + kn;
  k = kk + kpk;
  kpk_id = kpk;

  // L_o (2No x kk) and L_p = blkdiag of the holes' interpolation matrices
  Lo.alloc(std::max<size_t>(size_t(2) * No * kk, 1));
  Lo.zero(s);
  Lp.alloc(std::max<size_t>(size_t(2) * Np * kpk, 1));
  Lp.zero(s);
  std::vector<int> Jk, Jpk;
  {
    auto dfar = to_device_tmp(far_d, s), dnear = to_device_tmp(near_d, s);
    if (kf) gather_scatter(tf.P.p, int(far_d.size()), nullptr, Lo.p, 2 * No, dfar.p, int(far_d.size()), kf, s);
    if (kn) gather_scatter(tn.P.p, int(near_d.size()), nullptr, Lo.p + size_t(2) * No * kf, 2 * No, dnear.p,
                           int(near_d.size()), kn, s);
    std::vector<CopyProb> cp;
    int col = 0;
    for (int h = 0; h < nh; ++h) {
      const int m = 2 * (hoff[h + 1] - hoff[h]);
      if (tp[h].k) cp.push_back(CopyProb{tp[h].P.p, m, tp[h].k, m, Lp.p + 2 * size_t(hoff[h]) + size_t(col) * 2 * Np, 2 * Np});
      for (int i : tp[h].skel) Jpk.push_back(2 * hoff[h] + i);
      col += tp[h].k;
    }
    batched_copy(cp, s);
    RW_CUDA(cudaStreamSynchronize(s));
  }
  for (int i : tf.skel) Jk.push_back(far_d[i]);
  for (int i : tn.skel) Jk.push_back(near_d[i]);
  // a4, recompression (Sec. 3.4): a row ID of the skeleton block
  // R_k = A(J_k, I_p) (see recompress_rows; 960 columns, cheap).  The A_pk
  // blocks are not recompressed: their columns are every wall point, and
  // with P^div at hole_div_ratio = 4 hole radii (the wall points inside
  // taken explicitly) their ranks are already close to the blocks' own
  // (1920-panel channel, three holes: k_pk 505 -> 262 against 2 radii;
  // recompressing them as well gains 3 % of k for 30 % more time).
  const double rtol = 0.1 * ftol;
  if (recompress_enabled()) {
    IdMatProb ck{};
    ck.n2 = 2 * Np; ck.e2 = dall_p.p;
    recompress_rows(VW, Jk, ck, VW, true, VP, false, Lo, 2 * No, kk, rtol, o.seed + 404, s);
    k = kk + kpk;
    tr.mark("recompression");
  }
  // a5 (wall part): X_o = A_kk^{-1} L_o
  Xo.alloc(std::max<size_t>(size_t(2) * No * kk, 1));
  if (kk) solve_x(w.hbs, Lo.p, Xo.p, 2 * No, kk, s);
  auto dJk = to_device_tmp(Jk, s), dJpk = to_device_tmp(Jpk, s);
  Rkp.alloc(std::max<size_t>(size_t(kk) * 2 * Np, 1));
  Rpk.alloc(std::max<size_t>(size_t(kpk) * 2 * No, 1));
  eval_blocks({BlockProb{kk, 2 * Np, dJk.p, nullptr, 0, 0, 0, 1, 1.0, Rkp.p, kk},
               BlockProb{kpk, 2 * No, dJpk.p, nullptr, 0, 0, 1, 0, 1.0, Rpk.p, kpk}},
              VW, VP, s);
  tr.mark("L, R assembly, X_o");
  if (th1.joinable()) th1.join();
  RW_CUDA(cudaStreamSynchronize(s1));
  if (e1) std::rethrow_exception(e1);
  tr.mark("A_pp inverse (joined)");
  Xp.alloc(std::max<size_t>(size_t(2) * Np * kpk, 1));
  if (kpk) solve_x(hpp, Lp.p, Xp.p, 2 * Np, kpk, s);
  tr.mark("X_p = A_pp^-1 L_p");
  form_w(s);
  tr.mark("W, W^-1, solve program");
  bytes = Lo.bytes() + Lp.bytes() + Rkp.bytes() + Rpk.bytes() + Xo.bytes() + Xp.bytes() + Winv.bytes() + hpp.bytes +
          pn.buf.bytes() + nn.buf.bytes();
}

}  // namespace rw
