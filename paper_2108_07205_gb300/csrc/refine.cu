// Algorithm 1 (pre-computation and solve) for one local refinement.
//
// Ordering of the extended system: [o ; p] = the original points in panel
// order (kept and cut interleaved as on the wall) followed by the added
// points in window order.  A~ = blkdiag(A_oo, A_pp); the nonzero blocks of
// Q are -A_kc, A_kp (rows in I_k) and A_pk (rows in I_p) (Sec. 3.2).
//
// Low-rank factors (Sec. 3.3-3.4, uniform row-ID format: L = interpolation
// matrices, R = skeleton rows of A):
//  * far rows of I_k (outside P^div): one hierarchical ID against proxy
//    sources on P^bas, shared by A_kc and A_kp (Remark after Def. 3.1),
//    organised by the wall's own HBS tree (far_select / far_expand below);
//  * near rows of I_k: one direct ID of [A_kc^near | A_kp^near];
//  * A_pk: one hierarchical ID of the rows of [A_{p,div} | A_pk^near];
//  so L = blkdiag(L_k, L_pk) with L_k = [P_far ; P_near] on the k rows and
//  R = [[0, -A(J_k, I_c), A(J_k, I_p)], [A(J_pk, I_k), 0, 0]]: the row ID of
//  the blockwise factor L_1, whose kc and kp column blocks share their far
//  and near interpolation matrices (no duplicated columns).
//  Recompression (Sec. 3.4): the proxies stand for every possible source
//  near Gamma_r, so these ranks exceed those of the blocks themselves; row IDs
//  of the skeleton blocks R_k = [A(J_k, I_c), A(J_k, I_p)] and R_pk =
//  A(J_pk, I_k) (sketched when wide) fold into L and thin J (recompress_rows):
//  226 -> 81 on the 1024-panel channel (the paper's k_opt ~ 79, Sec. 3.4).
#include "refine.cuh"
#include <functional>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <exception>
#include <thread>

namespace rw {

namespace {

__global__ void k_identity(double* W, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x)
    W[e] = (e % n == e / n) ? 1.0 : 0.0;
}

// out[slot] = max(out[slot], max_j sum_i |A(i, j)|) for n x n column-major A:
// one warp per column; the maximum of non-negative doubles is taken on their
// bit patterns, which order the same way (out[slot] starts at 0).
__global__ void k_norm1(const double* A, int n, double* out, int slot) {
  const int lane = threadIdx.x & 31;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n) return;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += fabs(A[i + size_t(j) * n]);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(out + slot), static_cast<unsigned long long>(__double_as_longlong(s)));
}

__global__ void k_zero_cols(double* A, int ld, int nrows, const int* cols, int ncols) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nrows * ncols; e += gridDim.x * blockDim.x) {
    const int r = e % nrows, c = e / nrows;
    A[r + size_t(cols[c]) * ld] = 0.0;
  }
}

}  // namespace

// ---------------------------------------------------------------- far ID on the wall's tree
// The far-field rows of I_k against P^bas organised by the binary tree of the
// wall's own HBS (Sec. 3.3 allows the binary tree used in the HBS forward
// compression).  A node of the operator's HBS whose points are all far and
// whose proxy circle leaves every P^bas disk outside already has a row ID of
// its interaction with everything outside that circle: A(I_t, out) ~
// U_t^full A(J_t, out), U_t^full the product of the nested U's down to its
// leaves.  Such nodes (the largest ones, found top-down) contribute their
// skeleton rows J_t, the far points of the remaining leaves contribute
// themselves; one tree ID of these candidates against P^bas gives
// A(cand, I_r) ~ P A(J, I_r), and the far block of L_o is U^full P (raw
// candidates: the rows of P), formed top-down with P's right factor applied
// first.  The per-step work then scales with the number of candidates
// (about the skeletons of O(log N) nodes) instead of every far row.
struct FarOnTree {
  TreeId top;
  std::vector<int> cand;          // candidate DOFs: selected skeletons and raw far rows, in curve order
  std::vector<int> sel, sel_pos;  // selected heap nodes and the offset of their skeleton in cand
  std::vector<int> raw_dof, raw_pos;
};

// RW_FAR_ON_TREE=0 (diagnostics): the far-field ID over every far row in
// chunks of 128 instead.
bool far_on_tree_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("RW_FAR_ON_TREE");
    return !(e && e[0] == '0');
  }();
  return on;
}

namespace {

// Candidate selection.  isfar: per wall point; circ: (cx, cy, R) of each
// region's P^bas.  Node centres are the exact centroids; radii are bounded
// from the children up (a circle around both children's circles), which can
// only enlarge a proxy circle and so only makes the test stricter.
void far_select(const Hbs& H, const Wall& w, const std::vector<char>& isfar, const std::vector<double>& circ,
                FarOnTree& f) {
  const int L = H.L, nh = 2 << L;
  std::vector<double> cx(nh, 0.0), cy(nh, 0.0), rad(nh, 0.0);
  for (int h = 1 << L; h < nh; ++h) {
    const HbsNode& nd = H.node[h];
    double x = 0, y = 0;
    for (int i = nd.lo; i < nd.hi; ++i) { x += w.nodes.hx[i]; y += w.nodes.hy[i]; }
    const int n = std::max(nd.hi - nd.lo, 1);
    x /= n;
    y /= n;
    double r2 = 0;
    for (int i = nd.lo; i < nd.hi; ++i)
      r2 = std::max(r2, (w.nodes.hx[i] - x) * (w.nodes.hx[i] - x) + (w.nodes.hy[i] - y) * (w.nodes.hy[i] - y));
    cx[h] = x; cy[h] = y; rad[h] = std::sqrt(r2);
  }
  for (int h = (1 << L) - 1; h >= 1; --h) {
    const int a = 2 * h, b = 2 * h + 1;
    const double na = H.node[a].hi - H.node[a].lo, nb = H.node[b].hi - H.node[b].lo;
    cx[h] = (na * cx[a] + nb * cx[b]) / std::max(na + nb, 1.0);
    cy[h] = (na * cy[a] + nb * cy[b]) / std::max(na + nb, 1.0);
    rad[h] = std::max(std::hypot(cx[a] - cx[h], cy[a] - cy[h]) + rad[a],
                      std::hypot(cx[b] - cx[h], cy[b] - cy[h]) + rad[b]);
  }
  std::vector<int> pf(w.nodes.n + 1, 0);
  for (int i = 0; i < w.nodes.n; ++i) pf[i + 1] = pf[i] + (isfar[i] ? 1 : 0);
  const double ratio = w.opts.proxy_ratio;  // the proxy circles of the HBS compression
  std::function<void(int, int)> visit = [&](int h, int l) {
    const HbsNode& nd = H.node[h];
    const bool allfar = nd.hi > nd.lo && pf[nd.hi] - pf[nd.lo] == nd.hi - nd.lo;
    bool clear = allfar && l >= 1 && nd.k > 0;
    for (size_t r = 0; clear && r + 3 <= circ.size(); r += 3) {
      const double d = std::hypot(cx[h] - circ[r], cy[h] - circ[r + 1]);
      clear = d > (1.0 + 1e-9) * (ratio * rad[h] + circ[r + 2]);
    }
    if (clear) {
      f.sel.push_back(h);
      f.sel_pos.push_back(int(f.cand.size()));
      f.cand.insert(f.cand.end(), nd.skr.begin(), nd.skr.end());
      return;
    }
    if (l == L) {
      for (int i = nd.lo; i < nd.hi; ++i)
        if (isfar[i])
          for (int c = 0; c < 2; ++c) {
            f.raw_dof.push_back(2 * i + c);
            f.raw_pos.push_back(int(f.cand.size()));
            f.cand.push_back(2 * i + c);
          }
      return;
    }
    visit(2 * h, l + 1);
    visit(2 * h + 1, l + 1);
  };
  visit(1, 0);
}

// Rows of L_o (ld ldl) for the far rows: Pc (m_c x k2, ld m_c) is the top
// ID's interpolation matrix times the recompression's right factor.
void far_expand(const Hbs& H, const FarOnTree& f, const double* Pc, int k2, double* Lo, int ldl, cudaStream_t s) {
  const int mc = int(f.cand.size());
  if (!f.raw_dof.empty()) {
    auto dpos = to_device_tmp(f.raw_pos, s), ddof = to_device_tmp(f.raw_dof, s);
    gather_scatter(Pc, mc, dpos.p, Lo, ldl, ddof.p, int(f.raw_dof.size()), k2, s);
    RW_CUDA(cudaStreamSynchronize(s));
  }
  // down the tree: Y_t (k_t x k2) -> [Y_a; Y_b] = U_t Y_t; leaves -> L_o
  struct Act { int h, l; const double* Y; int ldy; };
  std::vector<Act> act;
  auto level_of = [](int h) { int l = 0; while (h > 1) { h >>= 1; ++l; } return l; };
  for (size_t q = 0; q < f.sel.size(); ++q) act.push_back(Act{f.sel[q], level_of(f.sel[q]), Pc + f.sel_pos[q], mc});
  std::vector<DBuf<double>> keep;
  while (!act.empty()) {
    size_t sz = 0;
    for (const Act& a : act) if (a.l < H.L) sz += size_t(H.node[a.h].m) * k2;
    DBuf<double> buf(std::max<size_t>(sz, 1));
    std::vector<GemmProb> gm;
    std::vector<Act> nxt;
    size_t off = 0;
    for (const Act& a : act) {
      const HbsNode& nd = H.node[a.h];
      const Hbs::Level& LV = H.lev[a.l];
      const int t = a.h - (1 << a.l);
      if (a.l == H.L) {
        const int n = 2 * (nd.hi - nd.lo);
        gm.push_back(GemmProb{LV.U.p + LV.oU[t], a.Y, Lo + 2 * size_t(nd.lo), n, k2, nd.k, n, a.ldy, ldl, 0, 0, 1.0, 0.0});
      } else {
        double* C = buf.p + off;
        gm.push_back(GemmProb{LV.U.p + LV.oU[t], a.Y, C, nd.m, k2, nd.k, nd.m, a.ldy, nd.m, 0, 0, 1.0, 0.0});
        const int ka = H.node[2 * a.h].k;
        nxt.push_back(Act{2 * a.h, a.l + 1, C, nd.m});
        nxt.push_back(Act{2 * a.h + 1, a.l + 1, C + ka, nd.m});
        off += size_t(nd.m) * k2;
      }
    }
    batched_gemm(gm, s);
    keep.push_back(std::move(buf));
    act = nxt;
  }
  RW_CUDA(cudaStreamSynchronize(s));  // the level buffers are released here
}

}  // namespace

bool recompress_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("RW_RECOMPRESS");
    return !(e && e[0] == '0');
  }();
  return on;
}

void recompress_rows(const NodesView& S, std::vector<int>& J, const IdMatProb& cols, const NodesView& E1, bool e1s,
                     const NodesView& E2, bool e2s, DBuf<double>& L, int m, int& k, double tol,
                     unsigned long long seed, cudaStream_t s) {
  if (k == 0 || J.empty()) return;
  IdMatProb cs = cols;
  cs.M = 0;
  cs.normal = 0;
  cs.ncirc = 0;
  cs.circ = nullptr;
  const Opts o;
  TreeId t = tree_row_id(S, J, cs, E1, e1s, E2, e2s, tol, o.sketch_cols, o.sketch_width, seed, 128, s);
  if (t.k >= k) return;
  DBuf<double> L2(std::max<size_t>(size_t(m) * t.k, 1));
  if (t.k) batched_gemm({GemmProb{L.p, t.P.p, L2.p, m, t.k, k, m, k, m, 0, 0, 1.0, 0.0}}, s);
  L = std::move(L2);
  std::vector<int> J2;
  for (int i : t.skel) J2.push_back(J[i]);
  J = J2;
  k = t.k;
}

void Wall::build_hbs(cudaStream_t s) {
  hbs.build(nodes, opts, s);
  hbs.make_fp32(s);
  hbs.make_bf16(s);
  if (opts.factor_tol() < opts.id_tol) {
    Opts oo = opts;
    oo.id_tol = opts.factor_tol();
    hbs_op.build(nodes, oo, s, true);
  }
  RW_CUDA(cudaStreamSynchronize(s));
}

SideStreams::~SideStreams() {
  // every buffer of the refinement has been released (stream ordered) by now
  for (cudaStream_t t : {s1, s2, s3}) if (t) { cudaStreamSynchronize(t); cudaStreamDestroy(t); }
}

Refinement::~Refinement() {
  // order the frees on the side streams after all work queued on the main
  // stream (the members are released after this body, the streams last)
  if (streams.main && (streams.s1 || streams.s2 || streams.s3)) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(ev, streams.main);
      if (streams.s1) cudaStreamWaitEvent(streams.s1, ev, 0);
      if (streams.s2) cudaStreamWaitEvent(streams.s2, ev, 0);
      if (streams.s3) cudaStreamWaitEvent(streams.s3, ev, 0);
      cudaEventDestroy(ev);
    }
  }
}

void Refinement::factor(const Wall& w, const std::vector<int>& pan, const std::vector<int>& lvl, cudaStream_t s,
                        const std::vector<double>* added) {
  wall = &w;
  streams.main = s;
  AllocStreamScope alloc_scope(s);
  Trace tr(s, "refine");
  const Opts& o = w.opts;
  // IDs (and A_pp) at the operator tolerance when that is tighter: the
  // factors then serve as the accurate operator for residuals as well
  const double ftol = o.factor_tol();
  const int P = w.n_panels;
  require(!pan.empty() && pan.size() == lvl.size(), "refine: need one level per cut panel");
  require(int(pan.size()) < P, "refine: cannot cut every panel");
  std::vector<char> cut(P, 0);
  // regions: maximal contiguous runs (mod P) of consecutive entries; several
  // regions grouped in one refinement share one factorisation of Q (Sec. 5.3,
  // the Remark on grouping refined regions)
  std::vector<int> rstart;
  for (size_t i = 0; i < pan.size(); ++i) {
    require(pan[i] >= 0 && pan[i] < P, "refine: panel id out of range");
    require(!cut[pan[i]], "refine: cut panels must be distinct");
    require(lvl[i] >= 0 && lvl[i] <= 12, "refine: level must be in 0..12");
    if (i == 0 || pan[i] != (pan[i - 1] + 1) % P) rstart.push_back(int(i));
    cut[pan[i]] = 1;
  }
  require(rstart.size() <= 8, "refine: at most 8 regions (contiguous runs of cut panels) per refinement");
  rstart.push_back(int(pan.size()));
  const int nreg = int(rstart.size()) - 1;
  panels = pan;
  levels = lvl;
  No = w.nodes.n;
  Ic.clear();
  Ik.clear();
  for (int j = 0; j < P; ++j)
    for (int q = 0; q < 16; ++q) (cut[j] ? Ic : Ik).push_back(16 * j + q);
  Nc = int(Ic.size());
  Nk = int(Ik.size());

  // a1: added nodes (window order)
  std::vector<double> ta, tb;
  std::vector<int> pstart(P, -1);
  const double h = 2.0 * kPi / P;
  int np = 0;
  for (size_t i = 0; i < pan.size(); ++i) {
    const int ns = 1 << lvl[i];
    pstart[pan[i]] = np;
    for (int q = 0; q < ns; ++q) {
      ta.push_back(pan[i] * h + q * (h / ns));
      tb.push_back(pan[i] * h + (q + 1) * (h / ns));
    }
    np += 16 * ns;
  }
  Np = np;
  Nn = Nk + Np;
  require(added || w.curve.kind != RW_CURVE_NODES,
          "refine: this wall was built from nodes; the added nodes must be given");
  const bool ext = w.nodes.kind == kNodesExterior;
  require(!ext || !added, "refine: an exterior wall's added nodes are evaluated on its curve");
  if (added) {
    // the caller's nodes for the sub-panels (window order)
    require(added->size() == size_t(6) * Np, "refine: added nodes do not match the cut panels and levels");
    pn.alloc(Np);
    RW_CUDA(cudaMemcpyAsync(pn.buf.p, added->data(), added->size() * sizeof(double), cudaMemcpyHostToDevice, s));
    pn.hx.assign(added->begin(), added->begin() + Np);
    pn.hy.assign(added->begin() + Np, added->begin() + 2 * size_t(Np));
  } else {
    auto dta = to_device_tmp(ta, s), dtb = to_device_tmp(tb, s);
    pn.alloc(Np);
    eval_nodes(w.curve, dta.p, dtb.p, int(ta.size()), pn.buf.p, Np, s);
    auto all = pn.buf.download(s);
    pn.hx.assign(all.begin(), all.begin() + Np);
    pn.hy.assign(all.begin() + Np, all.begin() + 2 * Np);
    if (ext) set_exterior_panels(pn, w.curve, ta, tb, s);
  }
  // refined order maps
  {
    std::vector<int> from_o, to_o, from_p, to_p, pts_o_src, pts_o_dst, pts_p_src, pts_p_dst;
    int in = 0;
    for (int j = 0; j < P; ++j) {
      if (!cut[j]) {
        for (int q = 0; q < 16; ++q, ++in) {
          pts_o_src.push_back(16 * j + q); pts_o_dst.push_back(in);
          for (int a = 0; a < 2; ++a) { from_o.push_back(2 * in + a); to_o.push_back(2 * (16 * j + q) + a); }
        }
      } else {
        int ns = 0;
        for (size_t i = 0; i < pan.size(); ++i) if (pan[i] == j) ns = 16 << lvl[i];
        for (int q = 0; q < ns; ++q, ++in) {
          pts_p_src.push_back(pstart[j] + q); pts_p_dst.push_back(in);
          for (int a = 0; a < 2; ++a) { from_p.push_back(2 * in + a); to_p.push_back(2 * (pstart[j] + q) + a); }
        }
      }
    }
    n_from_o = to_device(from_o, s); n_to_o = to_device(to_o, s);
    n_from_p = to_device(from_p, s); n_to_p = to_device(to_p, s);
    nko = int(from_o.size());
    nkp = int(from_p.size());
    nn.alloc(Nn);
    auto so = to_device_tmp(pts_o_src, s), dso = to_device_tmp(pts_o_dst, s);
    auto sp = to_device_tmp(pts_p_src, s), dsp = to_device_tmp(pts_p_dst, s);
    gather_scatter(w.nodes.buf.p, No, so.p, nn.buf.p, Nn, dso.p, int(pts_o_src.size()), 6, s);
    gather_scatter(pn.buf.p, Np, sp.p, nn.buf.p, Nn, dsp.p, int(pts_p_src.size()), 6, s);
    if (ext) {
      // the refined order's panels: kept panels, each cut one by its sub-panels
      std::vector<double> na, nb;
      for (int j = 0; j < P; ++j) {
        int ns = 1;
        for (size_t i = 0; i < pan.size(); ++i) if (pan[i] == j) ns = 1 << lvl[i];
        for (int q = 0; q < ns; ++q) { na.push_back(j * h + q * (h / ns)); nb.push_back(j * h + (q + 1) * (h / ns)); }
      }
      set_exterior_panels(nn, w.curve, na, nb, s);
    }
    std::vector<int> dcv;
    for (int i : Ic) { dcv.push_back(2 * i); dcv.push_back(2 * i + 1); }
    dc = to_device(dcv, s);
    RW_CUDA(cudaStreamSynchronize(s));
  }
  tr.mark("nodes+maps");
  // Gamma_r: centre and radius of the cut and added points
  // per region r: centre and radius rho_r of its cut and added points,
  // P^div (div_ratio rho_r) and P^bas (bas_ratio rho_r); kept points inside
  // any P^div are near, the rest far
  std::vector<int> poff(nreg + 1, 0);
  for (int r = 0; r < nreg; ++r) {
    int cnt = 0;
    for (int i = rstart[r]; i < rstart[r + 1]; ++i) cnt += 16 << lvl[i];
    poff[r + 1] = poff[r] + cnt;
  }
  std::vector<double> circ_div, circ_bas;
  for (int r = 0; r < nreg; ++r) {
    std::vector<int> pts;  // wall points cut by this region
    for (int i = rstart[r]; i < rstart[r + 1]; ++i)
      for (int q = 0; q < 16; ++q) pts.push_back(16 * pan[i] + q);
    double cx = 0, cy = 0;
    for (int i : pts) { cx += w.nodes.hx[i]; cy += w.nodes.hy[i]; }
    for (int i = poff[r]; i < poff[r + 1]; ++i) { cx += pn.hx[i]; cy += pn.hy[i]; }
    const double cnt = double(pts.size() + (poff[r + 1] - poff[r]));
    cx /= cnt;
    cy /= cnt;
    double rho2 = 0;
    for (int i : pts) rho2 = std::max(rho2, (w.nodes.hx[i] - cx) * (w.nodes.hx[i] - cx) + (w.nodes.hy[i] - cy) * (w.nodes.hy[i] - cy));
    for (int i = poff[r]; i < poff[r + 1]; ++i)
      rho2 = std::max(rho2, (pn.hx[i] - cx) * (pn.hx[i] - cx) + (pn.hy[i] - cy) * (pn.hy[i] - cy));
    const double rho = std::sqrt(rho2);
    circ_div.insert(circ_div.end(), {cx, cy, o.div_ratio * rho});
    circ_bas.insert(circ_bas.end(), {cx, cy, o.bas_ratio * rho});
  }
  // Exterior walls: a kept panel that shares a singular-rule pair with a cut
  // panel or an added sub-panel of region r is near r as well (its entries
  // against them are not the smooth kernel's that the proxies stand for)
  std::vector<char> ext_near_r;  // P x nreg
  if (ext) {
    ext_near_r.assign(size_t(P) * nreg, 0);
    for (int j = 0; j < P; ++j) {
      if (cut[j]) continue;
      const double tmj = w.nodes.htm[16 * j], thj = w.nodes.hth[16 * j];
      for (int r = 0; r < nreg; ++r) {
        bool hit = false;
        for (int i = rstart[r]; i < rstart[r + 1] && !hit; ++i)
          hit = ext_panels_interact(tmj, thj, w.nodes.htm[16 * pan[i]], w.nodes.hth[16 * pan[i]]);
        for (int q = poff[r]; q < poff[r + 1] && !hit; q += 16)
          hit = ext_panels_interact(tmj, thj, pn.htm[q], pn.hth[q]);
        ext_near_r[size_t(j) * nreg + r] = hit;
      }
    }
  }
  std::vector<int> far_d, near_d;
  std::vector<std::vector<int>> near_r(nreg);
  for (int i : Ik) {
    bool near = false;
    for (int r = 0; r < nreg; ++r) {
      const double dx = w.nodes.hx[i] - circ_div[3 * r], dy = w.nodes.hy[i] - circ_div[3 * r + 1];
      if (dx * dx + dy * dy < circ_div[3 * r + 2] * circ_div[3 * r + 2] ||
          (ext && ext_near_r[size_t(i / 16) * nreg + r])) {
        near = true;
        near_r[r].push_back(2 * i);
        near_r[r].push_back(2 * i + 1);
      }
    }
    auto& v = near ? near_d : far_d;
    v.push_back(2 * i);
    v.push_back(2 * i + 1);
  }

  // a2 and a3 are independent: A_pp^{-1} (dense below the threshold: a
  // single-leaf HBS is the dense inverse), the far-field ID and the near and
  // A_pk IDs run concurrently on three streams driven by three host threads.
  const NodesView VW = w.nodes.view(), VP = pn.view();
  TreeId tf, tn;
  FarOnTree ft;
  const bool use_tree = far_on_tree_enabled();
  DBuf<int> dall_p;
  std::vector<DBuf<int>> dnear_r(nreg);
  DBuf<double> dcirc_bas;
  {
    std::vector<int> pd(2 * Np);
    for (int i = 0; i < 2 * Np; ++i) pd[i] = i;
    dall_p = to_device(pd, s);
    for (int r = 0; r < nreg; ++r) dnear_r[r] = to_device(near_r[r], s);
    dcirc_bas = to_device(circ_bas, s);
    RW_CUDA(cudaStreamSynchronize(s));
  }
  RW_CUDA(cudaStreamCreateWithFlags(&streams.s1, cudaStreamNonBlocking));
  RW_CUDA(cudaStreamCreateWithFlags(&streams.s2, cudaStreamNonBlocking));
  RW_CUDA(cudaStreamCreateWithFlags(&streams.s3, cudaStreamNonBlocking));
  cudaStream_t s1 = streams.s1, s2 = streams.s2, s3 = streams.s3;
  std::exception_ptr e1, e2, e3;
  const bool recompress = recompress_enabled();
  const double rtol = 0.1 * ftol;  // recompression tolerance (see recompress_rows)
  // RW_SERIAL_REFINE=1 (diagnostics): run the four tasks one after another
  const char* ser = std::getenv("RW_SERIAL_REFINE");
  const bool serial = ser && ser[0] == '1';
  auto task1 = [&] {
    AllocStreamScope scope1(s1);
    try {
      Opts opp = o;
      pp_dense = Np <= o.dense_pp_max_points;
      opp.id_tol = ftol;
      if (pp_dense) opp.leaf_points = Np;
      hpp.build(pn, opp, s1);
      hpp.own_stream = s;   // later copies and programs live on the refinement's stream
      hpp.make_fp32(s1);
      hpp.make_bf16(s1);
      RW_CUDA(cudaStreamSynchronize(s1));
    } catch (...) { e1 = std::current_exception(); }
  };
  auto task2 = [&] {
    AllocStreamScope scope2(s2);
    try {
      // far rows of I_k against P^bas (shared by A_kc and A_kp); with several
      // regions against the union of their P^bas circles (every source lies
      // inside its own region's circle, every far row outside all of them)
      IdMatProb cs{};
      cs.cx = circ_bas[0]; cs.cy = circ_bas[1]; cs.R = circ_bas[2]; cs.M = o.n_proxy_refine; cs.normal = ext ? 0 : 1;
      if (nreg > 1) { cs.ncirc = nreg; cs.circ = dcirc_bas.p; }
      if (use_tree) {
        std::vector<char> isfar(w.nodes.n, 0);
        for (size_t q = 0; q < far_d.size(); q += 2) isfar[far_d[q] / 2] = 1;
        far_select(w.op(), w, isfar, circ_bas, ft);
        ft.top = tree_row_id(VW, ft.cand, cs, VW, true, VW, true, ftol, o.sketch_cols, o.sketch_width, o.seed + 101,
                             128, s2, true);
      } else {
        tf = tree_row_id(VW, far_d, cs, VW, true, VW, true, ftol, o.sketch_cols, o.sketch_width, o.seed + 101, 128,
                         s2, true);
      }
    } catch (...) { e2 = std::current_exception(); }
  };
  // A_pk: rows of [A_{p,div} | A_pk^near | n_p], then (recompression) a row
  // ID of R_pk = A(J_pk, I_k); needs neither the far nor the near ID
  std::vector<int> Jpk;
  auto task3 = [&] {
    AllocStreamScope scope3(s3);
    try {
      // region by region (its added rows against its P^div circle and the
      // kept points inside it): L_pk block diagonal over the regions
      std::vector<TreeId> tp(nreg);
      kpk = 0;
      for (int r = 0; r < nreg; ++r) {
        std::vector<int> prow;
        for (int d = 2 * poff[r]; d < 2 * poff[r + 1]; ++d) prow.push_back(d);
        IdMatProb cs{};
        cs.n1 = int(near_r[r].size()); cs.e1 = dnear_r[r].p;
        cs.cx = circ_div[3 * r]; cs.cy = circ_div[3 * r + 1]; cs.R = circ_div[3 * r + 2];
        cs.M = o.n_proxy_refine; cs.normal = ext ? 0 : 1;
        tp[r] = tree_row_id(VP, prow, cs, VW, false, VW, false, ftol, o.sketch_cols, o.sketch_width,
                            o.seed + 303 + 7 * r, 128, s3);
        kpk += tp[r].k;
      }
      kpk_id = kpk;
      if (nreg == 1) {
        Lp = std::move(tp[0].P);
        for (int i : tp[0].skel) Jpk.push_back(i);
      } else {
        Lp.alloc(std::max<size_t>(size_t(2) * Np * kpk, 1));
        Lp.zero(s3);
        std::vector<CopyProb> cp;
        int col = 0;
        for (int r = 0; r < nreg; ++r) {
          const int m = 2 * (poff[r + 1] - poff[r]);
          if (tp[r].k)
            cp.push_back(CopyProb{tp[r].P.p, m, tp[r].k, m, Lp.p + 2 * size_t(poff[r]) + size_t(col) * 2 * Np, 2 * Np});
          for (int i : tp[r].skel) Jpk.push_back(2 * poff[r] + i);
          col += tp[r].k;
        }
        batched_copy(cp, s3);
        RW_CUDA(cudaStreamSynchronize(s3));
      }
      if (recompress) {
        std::vector<int> kd;
        for (int i : Ik) { kd.push_back(2 * i); kd.push_back(2 * i + 1); }
        auto dkd = to_device_tmp(kd, s3);
        IdMatProb cp{};
        cp.n1 = int(kd.size()); cp.e1 = dkd.p;
        recompress_rows(VP, Jpk, cp, VW, false, VW, false, Lp, 2 * Np, kpk, rtol, o.seed + 505, s3);
      }
      // R_pk = A(J_pk, I_o) with the cut columns zeroed
      auto dJpk = to_device_tmp(Jpk, s3);
      Rpk.alloc(std::max<size_t>(size_t(kpk) * 2 * No, 1));
      eval_blocks({BlockProb{kpk, 2 * No, dJpk.p, nullptr, 0, 0, 1, 0, 1.0, Rpk.p, kpk}}, VW, VP, s3);
      if (kpk) {
        k_zero_cols<<<ceil_div((long long)kpk * 2 * Nc, 256), 256, 0, s3>>>(Rpk.p, kpk, kpk, dc.p, 2 * Nc);
        RW_CHECK_LAUNCH();
      }
      RW_CUDA(cudaStreamSynchronize(s3));
    } catch (...) { e3 = std::current_exception(); }
  };
  std::thread th1, th2, th3;
  // every exit from here on (including a throw) waits for the side threads
  struct Joiner {
    std::thread& t;
    ~Joiner() { if (t.joinable()) t.join(); }
  } join1{th1}, join2{th2}, join3{th3};
  if (serial) {
    task1();
    tr.mark("  A_pp inverse (HBS)");
    task2();
    tr.mark("  far ID");
    task3();
    tr.mark("  A_pk ID (+ recompression)");
  } else {
    th1 = std::thread(task1);
    th2 = std::thread(task2);
    th3 = std::thread(task3);
  }
  std::exception_ptr e0;
  try {
    // near rows of I_k: [A_kc^near | A_kp^near]
    IdMatProb cs{};
    cs.n1 = 2 * Nc; cs.e1 = dc.p; cs.n2 = 2 * Np; cs.e2 = dall_p.p; cs.M = 0; cs.normal = 0;
    tn = tree_row_id(VW, near_d, cs, VW, true, VP, false, ftol, o.sketch_cols, o.sketch_width, o.seed + 202, 128, s,
                     true);
  } catch (...) { e0 = std::current_exception(); }
  if (serial) tr.mark("  near ID");
  // X_o = A_oo^{-1} L_o needs only the far and near IDs: it runs on the main
  // stream while A_pp^{-1} may still be in construction on its own stream
  if (th2.joinable()) th2.join();
  RW_CUDA(cudaStreamSynchronize(s2));
  for (auto& e : {e0, e2}) if (e) std::rethrow_exception(e);
  tr.mark("IDs (concurrent with A_pp)");
  kf = use_tree ? ft.top.k : tf.k; kn = tn.k; kk = kf + kn;
  // skeleton DOFs
  std::vector<int> Jk;
  if (use_tree) for (int i : ft.top.skel) Jk.push_back(ft.cand[i]);
  else for (int i : tf.skel) Jk.push_back(far_d[i]);
  for (int i : tn.skel) Jk.push_back(near_d[i]);
  // Recompression (Sec. 3.4): a row ID of R_k = [A(J_k, I_c), A(J_k, I_p)]
  // whose interpolation matrix T (kk x k2) multiplies L_o = [P_far ; P_near]
  // (block columns kf | kn, disjoint rows) from the right.  It needs only
  // the skeletons, so it runs before L_o exists, and the far and near trees
  // are expanded into P_far T(0:kf, :) and P_near T(kf:kk, :) directly.
  TreeId rk;
  bool reduced = false;
  if (recompress && kk > 0) {
    IdMatProb ck{};
    ck.n1 = 2 * Nc; ck.e1 = dc.p; ck.n2 = 2 * Np; ck.e2 = dall_p.p;
    rk = tree_row_id(VW, Jk, ck, VW, true, VP, false, rtol, o.sketch_cols, o.sketch_width, o.seed + 404, 128, s);
    reduced = rk.k < kk;
    tr.mark("recompression (wall rows)");
  }
  const int k2 = reduced ? rk.k : kk;
  // L_o (2No x k2)
  Lo.alloc(std::max<size_t>(size_t(2) * No * k2, 1));
  Lo.zero(s);
  {
    auto dfar = to_device_tmp(far_d, s), dnear = to_device_tmp(near_d, s);
    const double* T = reduced ? rk.P.p : nullptr;
    if (kf && k2 && use_tree) {
      const int kout = reduced ? k2 : kf;
      DBuf<double> Pc = ft.top.expand(T, kk, kout, s);
      far_expand(w.op(), ft, Pc.p, kout, Lo.p, 2 * No, s);
    } else if (kf && k2) {
      DBuf<double> Pf = tf.expand(T, kk, k2, s);
      gather_scatter(Pf.p, int(far_d.size()), nullptr, Lo.p, 2 * No, dfar.p, int(far_d.size()), reduced ? k2 : kf, s);
      RW_CUDA(cudaStreamSynchronize(s));
    }
    if (kn && k2) {
      DBuf<double> Pn = tn.expand(T ? T + kf : nullptr, kk, k2, s);
      double* dst = reduced ? Lo.p : Lo.p + size_t(2) * No * kf;
      gather_scatter(Pn.p, int(near_d.size()), nullptr, dst, 2 * No, dnear.p, int(near_d.size()), reduced ? k2 : kn, s);
      RW_CUDA(cudaStreamSynchronize(s));
    }
  }
  if (reduced) {
    std::vector<int> J2;
    for (int i : rk.skel) J2.push_back(Jk[i]);
    Jk = J2;
  }
  kk = k2;
  tr.mark("L_o (deferred expansion)");
  if (th3.joinable()) th3.join();
  if (e3) std::rethrow_exception(e3);
  k = kk + kpk;
  // a5 (o part): X_o = A_oo^{-1} L_o
  Xo.alloc(std::max<size_t>(size_t(2) * No * kk, 1));
  if (kk) solve_x(w.hbs, Lo.p, Xo.p, 2 * No, kk, s);
  auto dJk = to_device_tmp(Jk, s);
  Rkc.alloc(std::max<size_t>(size_t(kk) * 2 * Nc, 1));
  Rkp.alloc(std::max<size_t>(size_t(kk) * 2 * Np, 1));
  eval_blocks({BlockProb{kk, 2 * Nc, dJk.p, dc.p, 0, 0, 0, 0, -1.0, Rkc.p, kk},
               BlockProb{kk, 2 * Np, dJk.p, nullptr, 0, 0, 0, 1, 1.0, Rkp.p, kk}},
              VW, VP, s);
  tr.mark("L, R assembly, X_o");
  // a5 (p part): X_p = A_pp^{-1} L_p once A_pp^{-1} is built
  if (th1.joinable()) th1.join();
  RW_CUDA(cudaStreamSynchronize(s1));
  if (e1) std::rethrow_exception(e1);
  tr.mark("A_pp inverse (joined)");
  Xp.alloc(std::max<size_t>(size_t(2) * Np * kpk, 1));
  if (kpk) solve_x(hpp, Lp.p, Xp.p, 2 * Np, kpk, s);
  tr.mark("X_p = A_pp^-1 L_p");
  form_w(s);
  tr.mark("W, W^-1, solve program");
  bytes = Lo.bytes() + Lp.bytes() + Rkc.bytes() + Rkp.bytes() + Rpk.bytes() + Xo.bytes() + Xp.bytes() + Winv.bytes() +
          hpp.bytes + pn.buf.bytes() + nn.buf.bytes();
}

namespace {
__global__ void k_d2f_x(const double* in, float* out, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    out[i] = float(in[i]);
}
__global__ void k_f2d_x(const float* in, double* out, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    out[i] = double(in[i]);
}
}  // namespace

void Refinement::solve_x(const Hbs& H, const double* L, double* X, int m, int kc, cudaStream_t s) const {
  if (!wall->opts.mixed_factor) {
    H.apply_inverse_levels(L, X, kc, s);
    return;
  }
  if (wall->opts.mixed_factor == 2) {  // double-FP32 sweeps, one launch per 64 columns
    H.inverse_gemm_df(L, X, kc, s);
    return;
  }
  // FP32 sweeps: X serves the preconditioner only (W is formed from it in FP64)
  const size_t n = size_t(m) * kc;
  TBuf<float> l32(n, s), x32(n, s);
  const int grid = int(std::min<size_t>((n + 255) / 256, 4096));
  k_d2f_x<<<grid, 256, 0, s>>>(L, l32.p, n);
  RW_CHECK_LAUNCH();
  H.apply_inverse_f32(l32.p, x32.p, kc, s);
  k_f2d_x<<<grid, 256, 0, s>>>(x32.p, X, n);
  RW_CHECK_LAUNCH();
}

void Refinement::form_w(cudaStream_t s) {
  TBuf<double> W(size_t(k) * k, s), Ww(size_t(k) * k, s), Xc(size_t(2) * Nc * std::max(kk, 1), s);
  k_identity<<<ceil_div((long long)k * k, 256), 256, 0, s>>>(W.p, k);
  RW_CHECK_LAUNCH();
  if (kk && Nc) gather_scatter(Xo.p, 2 * No, dc.p, Xc.p, 2 * Nc, nullptr, 2 * Nc, kk, s);
  if (wall->opts.mixed_factor) {
    // a factorisation for the iterative modes: the products in double-FP32
    // (R held as FP32 pairs; the copies serve the solve programs later)
    AllocStreamScope scope(streams.main);
    for (auto pr : {std::make_pair(&Rkc, &Rkc2), std::make_pair(&Rkp, &Rkp2), std::make_pair(&Rpk, &Rpk2)}) {
      pr.second->alloc(pr.first->n);
      copy_d2df(pr.first->p, pr.second->p, pr.first->n, s);
    }
    std::vector<GemmDfProb> g;
    if (kk && Nc) g.push_back(GemmDfProb{Rkc2.p, Xc.p, W.p, kk, kk, 2 * Nc, kk, 2 * Nc, k, 1.0, 1.0});
    if (kk && kpk) g.push_back(GemmDfProb{Rkp2.p, Xp.p, W.p + size_t(kk) * k, kk, kpk, 2 * Np, kk, 2 * Np, k, 1.0, 1.0});
    if (kk && kpk) g.push_back(GemmDfProb{Rpk2.p, Xo.p, W.p + kk, kpk, kk, 2 * No, kpk, 2 * No, k, 1.0, 1.0});
    batched_gemm_df(g, s);
  } else {
    std::vector<GemmProb> g;
    if (kk && Nc) g.push_back(GemmProb{Rkc.p, Xc.p, W.p, kk, kk, 2 * Nc, kk, 2 * Nc, k, 0, 0, 1.0, 1.0});
    if (kk && kpk) g.push_back(GemmProb{Rkp.p, Xp.p, W.p + size_t(kk) * k, kk, kpk, 2 * Np, kk, 2 * Np, k, 0, 0, 1.0, 1.0});
    if (kk && kpk) g.push_back(GemmProb{Rpk.p, Xo.p, W.p + kk, kpk, kk, 2 * No, kpk, 2 * No, k, 0, 0, 1.0, 1.0});
    batched_gemm(g, s);
  }
  Winv.alloc(std::max<size_t>(size_t(k) * k, 1));
  DBuf<int> flag(1);
  DBuf<double> norms(2);
  flag.zero(s);
  norms.zero(s);
  if (k) {
    k_norm1<<<ceil_div(32LL * k, 256), 256, 0, s>>>(W.p, k, norms.p, 0);
    RW_CHECK_LAUNCH();
  }
  batched_inverse({InvProb{W.p, Winv.p, Ww.p, k, k, k, flag.p}}, s);
  if (k) {
    k_norm1<<<ceil_div(32LL * k, 256), 256, 0, s>>>(Winv.p, k, norms.p, 1);
    RW_CHECK_LAUNCH();
  }
  // the solve program depends on the buffers, not on their values: the host
  // builds it while the GPU forms W and W^-1 (the direct modes it serves
  // refuse a factorisation for the iterative modes)
  if (!wall->opts.mixed_factor) build_solve_program(s);
  auto hf = flag.download(s);
  require(hf[0] == 0, "refine: Woodbury operator W = I + R X is singular", RW_ERR_SINGULAR);
  const auto hn = norms.download(s);
  cond_w = hn[0] * hn[1];
}

void Refinement::woodbury_correct(double* yo, double* yp, int nrhs, cudaStream_t s) const {
  if (k == 0) return;
  TBuf<double> yc(size_t(2) * Nc * nrhs, s), r(size_t(k) * nrhs, s), z(size_t(k) * nrhs, s);
  if (Nc) gather_scatter(yo, 2 * No, dc.p, yc.p, 2 * Nc, nullptr, 2 * Nc, nrhs, s);
  // r = R y (with nothing cut, the k rows of R are R_kp alone)
  std::vector<GemvProb<double>> p1;
  if (kk && Nc) p1.push_back(GemvProb<double>{Rkc.p, yc.p, r.p, kk, 2 * Nc, kk, 2 * Nc, k, 1.0, 0.0});
  if (kpk) p1.push_back(GemvProb<double>{Rpk.p, yo, r.p + kk, kpk, 2 * No, kpk, 2 * No, k, 1.0, 0.0});
  matvec<double>(p1, nrhs, s);
  if (kk && Np)
    matvec<double>({GemvProb<double>{Rkp.p, yp, r.p, kk, 2 * Np, kk, 2 * Np, k, 1.0, Nc ? 1.0 : 0.0}}, nrhs, s);
  // z = W^{-1} r
  matvec<double>({GemvProb<double>{Winv.p, r.p, z.p, k, k, k, k, k, 1.0, 0.0}}, nrhs, s);
  // y -= X z
  std::vector<GemvProb<double>> p2;
  if (kk) p2.push_back(GemvProb<double>{Xo.p, z.p, yo, 2 * No, kk, 2 * No, k, 2 * No, -1.0, 1.0});
  if (kpk) p2.push_back(GemvProb<double>{Xp.p, z.p + kk, yp, 2 * Np, kpk, 2 * Np, k, 2 * Np, -1.0, 1.0});
  matvec<double>(p2, nrhs, s);
}

void Refinement::emit_solve(Program& P, int gb, long long g_off, int ldg, int tb, long long t_off, int ldt) const {
  const int WS = 2;  // workspace base (ld -1: per-RHS block)
  const long long go = P.ws_alloc(2LL * No), gp = P.ws_alloc(2LL * Np);
  const long long yo = P.ws_alloc(2LL * No), yp = P.ws_alloc(2LL * Np);
  P.zero(0, 2 * No, WS, go, -1, nullptr);
  P.copy(0, nkp, gb, g_off, ldg, n_from_p.p, WS, gp, -1, n_to_p.p);
  P.copy(1, nko, gb, g_off, ldg, n_from_o.p, WS, go, -1, n_to_o.p);
  const int pa = wall->hbs.emit_inverse_sweep(P, 2, WS, go, -1, WS, yo, -1);
  const int pb = hpp.emit_inverse_sweep(P, 2, WS, gp, -1, WS, yp, -1);
  int p = std::max(pa, pb);
  if (k > 0) {
    const long long yc = P.ws_alloc(std::max(2LL * Nc, 1LL)), r = P.ws_alloc(k), z = P.ws_alloc(k);
    if (Nc) {
      P.copy(p++, 2 * Nc, WS, yo, -1, dc.p, WS, yc, -1, nullptr);
      if (kk) P.gemv(p, Rkc.p, kk, 2 * Nc, kk, WS, yc, -1, WS, r, -1, 1.0, 0.0);
    }
    if (kpk) P.gemv(p, Rpk.p, kpk, 2 * No, kpk, WS, yo, -1, WS, r + kk, -1, 1.0, 0.0);
    if (kk && Np) P.gemv(p + 1, Rkp.p, kk, 2 * Np, kk, WS, yp, -1, WS, r, -1, 1.0, Nc ? 1.0 : 0.0);
    p += 2;
    P.gemv(p++, Winv.p, k, k, k, WS, r, -1, WS, z, -1, 1.0, 0.0);
    if (kk) P.gemv(p, Xo.p, 2 * No, kk, 2 * No, WS, z, -1, WS, yo, -1, -1.0, 1.0);
    if (kpk) P.gemv(p, Xp.p, 2 * Np, kpk, 2 * Np, WS, z + kk, -1, WS, yp, -1, -1.0, 1.0);
    ++p;
  }
  P.copy(p, nko, WS, yo, -1, n_to_o.p, tb, t_off, ldt, n_from_o.p);
  P.copy(p, nkp, WS, yp, -1, n_to_p.p, tb, t_off, ldt, n_from_p.p);
}

void Refinement::emit_to_ext(Program& P, int gb, long long g_off, int ldg, int eb, long long e_off, int lde) const {
  P.zero(0, 2 * No, eb, e_off, lde, nullptr);
  P.copy(0, nkp, gb, g_off, ldg, n_from_p.p, eb, e_off + 2LL * No, lde, n_to_p.p);
  P.copy(1, nko, gb, g_off, ldg, n_from_o.p, eb, e_off, lde, n_to_o.p);
}

void Refinement::emit_from_ext(Program& P, int eb, long long e_off, int lde, int tb, long long t_off, int ldt) const {
  P.copy(0, nko, eb, e_off, lde, n_to_o.p, tb, t_off, ldt, n_from_o.p);
  P.copy(0, nkp, eb, e_off + 2LL * No, lde, n_to_p.p, tb, t_off, ldt, n_from_p.p);
}

void Refinement::emit_ext_direct(Program& P, int vb, long long vo, int ldv, int yb, long long yo, int ldy) const {
  const int WS = 2;
  const long long vp = vo + 2LL * No, yp = yo + 2LL * No;
  const int pa = wall->hbs.emit_inverse_sweep(P, 0, vb, vo, ldv, yb, yo, ldy);
  const int pb = hpp.emit_inverse_sweep(P, 0, vb, vp, ldv, yb, yp, ldy);
  int p = std::max(pa, pb);
  if (k == 0) return;
  // r = R y, z = W^{-1} r, y -= X z (Eq. wood)
  const long long yc = P.ws_alloc(std::max(2LL * Nc, 1LL)), r = P.ws_alloc(k), z = P.ws_alloc(k);
  if (Nc) {
    P.copy(p++, 2 * Nc, yb, yo, ldy, dc.p, WS, yc, -1, nullptr);
    if (kk) P.gemv(p, Rkc.p, kk, 2 * Nc, kk, WS, yc, -1, WS, r, -1, 1.0, 0.0);
  }
  if (kpk) P.gemv(p, Rpk.p, kpk, 2 * No, kpk, yb, yo, ldy, WS, r + kk, -1, 1.0, 0.0);
  if (kk && Np) P.gemv(p + 1, Rkp.p, kk, 2 * Np, kk, yb, yp, ldy, WS, r, -1, 1.0, Nc ? 1.0 : 0.0);
  p += 2;
  P.gemv(p++, Winv.p, k, k, k, WS, r, -1, WS, z, -1, 1.0, 0.0);
  if (kk) P.gemv(p, Xo.p, 2 * No, kk, 2 * No, WS, z, -1, yb, yo, ldy, -1.0, 1.0);
  if (kpk) P.gemv(p, Xp.p, 2 * Np, kpk, 2 * Np, WS, z + kk, -1, yb, yp, ldy, -1.0, 1.0);
}

void Refinement::emit_ext_operator(Program& P, int xb, long long xo, int ldx, int yb, long long yo, int ldy) const {
  const int WS = 2;
  const long long xp = xo + 2LL * No, yp = yo + 2LL * No;
  const int pw = wall->op().emit_forward_sweep(P, 0, xb, xo, ldx, yb, yo, ldy);
  const int pp = hpp.emit_forward_sweep(P, 0, xb, xp, ldx, yb, yp, ldy);
  if (k == 0) return;
  // r = R x (phases 0-2), then y += L r once the sweeps are done
  const long long xc = P.ws_alloc(std::max(2LL * Nc, 1LL)), r = P.ws_alloc(k);
  if (Nc) P.copy(0, 2 * Nc, xb, xo, ldx, dc.p, WS, xc, -1, nullptr);
  if (kpk) P.gemv(0, Rpk.p, kpk, 2 * No, kpk, xb, xo, ldx, WS, r + kk, -1, 1.0, 0.0);
  if (kk && Nc) P.gemv(1, Rkc.p, kk, 2 * Nc, kk, WS, xc, -1, WS, r, -1, 1.0, 0.0);
  if (kk && Np) P.gemv(2, Rkp.p, kk, 2 * Np, kk, xb, xp, ldx, WS, r, -1, 1.0, Nc ? 1.0 : 0.0);
  const int q = std::max(3, std::max(pw, pp));
  if (kk) P.gemv(q, Lo.p, 2 * No, kk, 2 * No, WS, r, -1, yb, yo, ldy, 1.0, 1.0);
  if (kpk) P.gemv(q, Lp.p, 2 * Np, kpk, 2 * Np, WS, r + kk, -1, yb, yp, ldy, 1.0, 1.0);
}

void Refinement::build_solve_program(cudaStream_t s) {
  // bases: 0 = g (2Nn x nrhs), 1 = tau (2Nn x nrhs), 2 = workspace
  emit_solve(solve_prog, 0, 0, 2 * Nn, 1, 0, 2 * Nn);
  solve_prog.finalize(s);
}

void Refinement::solve_direct(const double* g, double* tau, int nrhs, cudaStream_t s) const {
  // Many right-hand sides: the level-by-level sweeps run as batched GEMMs,
  // which use the FP64 units better than 8-RHS chunks of the GEMV program
  // (64 RHS on the 2048-panel channel: 2x the solve rate).  RW_SOLVE_GEMM_RHS
  // (tuning) sets the smallest nrhs that takes them (default 16).
  static const int gemm_rhs = [] {
    const char* e = std::getenv("RW_SOLVE_GEMM_RHS");
    const int v = e ? std::atoi(e) : 0;
    return v > 0 ? v : 16;
  }();
  if (nrhs >= gemm_rhs) {
    solve_direct_levels(g, tau, nrhs, s);
    return;
  }
  require(!wall->opts.mixed_factor, "solve_direct: a factorisation for the iterative modes (opts.mixed_factor)");
  const size_t need = size_t(std::max<long long>(solve_prog.ws_per_rhs(), 1)) * nrhs;
  if (solve_ws.n < need) solve_ws.alloc(need);
  double* bases[kMaxBases] = {const_cast<double*>(g), tau, solve_ws.p, nullptr};
  solve_prog.run(bases, nrhs, s);
}

void Refinement::solve_direct_levels(const double* g, double* tau, int nrhs, cudaStream_t s) const {
  TBuf<double> go(size_t(2) * No * nrhs, s), gp(size_t(2) * Np * nrhs, s);
  TBuf<double> yo(size_t(2) * No * nrhs, s), yp(size_t(2) * Np * nrhs, s);
  fill_zero(go.p, go.n, s);
  gather_scatter(g, 2 * Nn, n_from_o.p, go.p, 2 * No, n_to_o.p, nko, nrhs, s);
  gather_scatter(g, 2 * Nn, n_from_p.p, gp.p, 2 * Np, n_to_p.p, nkp, nrhs, s);
  if (nrhs > 8) {
    // both trees and the Woodbury correction in one launch per 64 RHS
    run_prog(dir_prog(s), go.p, gp.p, yo.p, yp.p, (double*)nullptr, nrhs, s);
  } else {
    wall->hbs.apply_inverse_levels(go.p, yo.p, nrhs, s);
    hpp.apply_inverse_levels(gp.p, yp.p, nrhs, s);
    woodbury_correct(yo.p, yp.p, nrhs, s);
  }
  gather_scatter(yo.p, 2 * No, n_to_o.p, tau, 2 * Nn, n_from_o.p, nko, nrhs, s);
  gather_scatter(yp.p, 2 * Np, n_to_p.p, tau, 2 * Nn, n_from_p.p, nkp, nrhs, s);
}

void Refinement::solve_refined(const double* g, double* tau, int nrhs, int steps, cudaStream_t s) const {
  solve_direct(g, tau, nrhs, s);
  if (steps <= 0) return;
  const size_t n = size_t(2) * Nn * nrhs;
  TBuf<double> r(n, s), d(n, s);
  for (int it = 0; it < steps; ++it) {
    apply_nn(tau, r.p, nrhs, s);
    // r = g - A tau ; tau += A_ext^{-1} r
    axpby(g, r.p, n, 1.0, -1.0, s);
    solve_direct(r.p, d.p, nrhs, s);
    axpby(d.p, tau, n, 1.0, 1.0, s);
  }
}

void Refinement::apply_nn(const double* x, double* y, int nrhs, cudaStream_t s) const {
  if (nn.kind == kNodesExterior) {
    // exterior wall: blocks of rows of A_nn = 1/2 I + D + S evaluated (with
    // the singular rule) into a scratch matrix, each applied by a GEMM
    const int n = 2 * Nn;
    const int rb = std::max(2, std::min(n, int((size_t(1) << 25) / size_t(n)) & ~1));
    TBuf<double> T(size_t(rb) * n, s);
    const NodesView V = nn.view();
    for (int r0 = 0; r0 < n; r0 += rb) {
      const int m = std::min(rb, n - r0);
      eval_blocks({BlockProb{m, n, nullptr, nullptr, r0, 0, 0, 0, 1.0, T.p, m}}, V, V, s);
      batched_gemm({GemmProb{T.p, x, y + r0, m, nrhs, n, m, n, n, 0, 0, 1.0, 0.0}}, s);
    }
    return;
  }
  if (!holes) {
    apply_exact(nn.view(), x, y, nrhs, s);
    return;
  }
  // [y_k; y_p] = [A_kk x_k + A_kp x_p; A_pk x_k + A_pp x_p]; wall rows first
  const int ld = 2 * Nn, ko = 2 * No;
  const NodesView VW = wall->nodes.view(), VP = pn.view();
  apply_exact(VW, x, y, nrhs, s, ld, ld);
  apply_cross(VW, VP, x + ko, ld, y, ld, nrhs, true, s);
  apply_cross(VP, VW, x, ld, y + ko, ld, nrhs, false, s);
  matvec<double>({GemvProb<double>{hpp.lev[0].D.p, x + ko, y + ko, 2 * Np, 2 * Np, 2 * Np, ld, ld, 1.0, 1.0}}, nrhs, s);
}

void Refinement::velocity(const double* tau, int nrhs, int nt, const double* targets, double* u,
                          cudaStream_t s) const {
  if (!holes) {
    eval_velocity(nn.view(), tau, nrhs, nt, targets, u, s);
    return;
  }
  eval_velocity(wall->nodes.view(), tau, nrhs, nt, targets, u, s, 2 * Nn, false);
  eval_velocity(pn.view(), tau + 2 * No, nrhs, nt, targets, u, s, 2 * Nn, true);
}

void Refinement::pressure(const double* tau, int nrhs, int nt, const double* targets, double* p,
                          cudaStream_t s) const {
  if (!holes) {
    eval_pressure(nn.view(), tau, nrhs, nt, targets, p, s);
    return;
  }
  eval_pressure(wall->nodes.view(), tau, nrhs, nt, targets, p, s, 2 * Nn, false);
  eval_pressure(pn.view(), tau + 2 * No, nrhs, nt, targets, p, s, 2 * Nn, true);
}

void Refinement::apply_els(const double* xo, const double* xp, double* yo, double* yp, int nrhs, cudaStream_t s) const {
  if (nrhs > 8) {
    run_prog(els_prog(false, s), xo, xp, yo, yp, (double*)nullptr, nrhs, s);
    return;
  }
  wall->op().apply_forward(xo, yo, nrhs, s);
  hpp.apply_forward(xp, yp, nrhs, s);
  if (k == 0) return;
  TBuf<double> xc(size_t(2) * Nc * nrhs, s), r(size_t(k) * nrhs, s);
  if (Nc) gather_scatter(xo, 2 * No, dc.p, xc.p, 2 * Nc, nullptr, 2 * Nc, nrhs, s);
  std::vector<GemvProb<double>> p1;
  if (kk && Nc) p1.push_back(GemvProb<double>{Rkc.p, xc.p, r.p, kk, 2 * Nc, kk, 2 * Nc, k, 1.0, 0.0});
  if (kpk) p1.push_back(GemvProb<double>{Rpk.p, xo, r.p + kk, kpk, 2 * No, kpk, 2 * No, k, 1.0, 0.0});
  matvec<double>(p1, nrhs, s);
  if (kk && Np)
    matvec<double>({GemvProb<double>{Rkp.p, xp, r.p, kk, 2 * Np, kk, 2 * Np, k, 1.0, Nc ? 1.0 : 0.0}}, nrhs, s);
  std::vector<GemvProb<double>> p2;
  if (kk) p2.push_back(GemvProb<double>{Lo.p, r.p, yo, 2 * No, kk, 2 * No, k, 2 * No, 1.0, 1.0});
  if (kpk) p2.push_back(GemvProb<double>{Lp.p, r.p + kk, yp, 2 * Np, kpk, 2 * Np, k, 2 * Np, 1.0, 1.0});
  matvec<double>(p2, nrhs, s);
}

}  // namespace rw
