// HBS construction, inversion and sweeps on the device (Gillman, Young and
// Martinsson 2012, as used by the paper for A_oo and, above the dense
// threshold, for A_pp).  Host code plans the tree and index sets; every
// matrix entry, factorisation and product is computed by the kernels in
// dense.cu / eval.cu.
#include "hbs.cuh"
#include <mutex>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <numeric>
#include <type_traits>

namespace rw {

// ====================================================================== IdBatch
int IdBatch::add(const IdMatProb& spec, int sketch_cols, int sketch_width) {
  Job j;
  j.spec = spec;
  j.spec.ncol = idmat_ncol(spec.kind, spec.n1, spec.n2, idmat_nproxy(spec), spec.normal, spec.sl_in);
  if (j.spec.ncol > sketch_cols && sketch_width < j.spec.ncol) {
    j.sk_width = sketch_width;
    j.nr = sketch_width;
  } else {
    j.nr = j.spec.ncol;
  }
  jobs.push_back(j);
  return int(jobs.size()) - 1;
}

void IdBatch::run(const NodesView& S, const NodesView& E1, bool e1s, const NodesView& E2, bool e2s,
                  double tol_rel, const std::vector<double>& tol_abs, const std::vector<int>& subset_in,
                  const std::vector<int>& min_rank, const std::vector<int>& max_rank,
                  unsigned long long seed, cudaStream_t s) {
  const int nj = int(jobs.size());
  if (!W.p) {
    size_t w = 0, m = 0, nm = 0;
    for (auto& j : jobs) {
      j.woff = w;
      j.moff = m;
      j.noff = nm;
      w += size_t(j.nr) * j.spec.m;
      m += j.spec.m;
      nm += id_norms_elems(j.spec.m);
    }
    W.alloc(std::max<size_t>(w, 1));
    norms.alloc(std::max<size_t>(nm, 1));
    piv.alloc(std::max<size_t>(m, 1));
    rank.alloc(std::max(nj, 1));
    h_rank.assign(nj, 0);
  }
  std::vector<int> subset = subset_in;
  if (subset.empty()) { subset.resize(nj); std::iota(subset.begin(), subset.end(), 0); }
  // evaluation: direct into W, or into Y followed by the sketch W = Omega^T Y
  size_t ysz = 0;
  int max_ncol = 0, max_sk = 0;
  for (int id : subset) {
    const Job& j = jobs[id];
    if (j.sk_width) {
      ysz += size_t(j.spec.ncol) * j.spec.m;
      max_ncol = std::max(max_ncol, j.spec.ncol);
      max_sk = std::max(max_sk, j.sk_width);
    }
  }
  TBuf<double> Y(ysz, s), Om(size_t(max_ncol) * max_sk, s);
  if (max_sk) fill_rademacher(Om.p, Om.n, seed, s);
  std::vector<IdMatProb> ev;
  std::vector<GemmProb> gm;
  size_t yo = 0;
  for (int id : subset) {
    Job& j = jobs[id];
    IdMatProb p = j.spec;
    if (j.sk_width) {
      p.W = Y.p + yo;
      p.ldw = p.ncol;
      GemmProb g{Om.p, p.W, W.p + j.woff, j.sk_width, p.m, p.ncol, max_ncol, p.ncol, j.sk_width, 1, 0, 1.0, 0.0};
      gm.push_back(g);
      yo += size_t(p.ncol) * p.m;
    } else {
      p.W = W.p + j.woff;
      p.ldw = p.ncol;
    }
    ev.push_back(p);
  }
  eval_idmat(ev, S, E1, e1s, E2, e2s, s);
  batched_gemm(gm, s);
  std::vector<IdProb> ip;
  for (int id : subset) {
    Job& j = jobs[id];
    IdProb q{};
    q.W = W.p + j.woff;
    q.ldw = j.nr;
    q.nr = j.nr;
    q.nc = j.spec.m;
    q.tol_abs = tol_abs.empty() ? 0.0 : tol_abs[id];
    q.tol_rel = tol_rel;
    q.min_rank = min_rank.empty() ? 0 : min_rank[id];
    q.max_rank = max_rank.empty() ? j.spec.m : max_rank[id];
    q.piv = piv.p + j.moff;
    q.norms = norms.p + j.noff;
    q.P = nullptr;
    q.ldp = j.spec.m;
    q.rank = rank.p + id;
    ip.push_back(q);
  }
  batched_id(ip, s, paired && subset_in.empty());
  h_rank = rank.download(s);
  h_rank.resize(nj);
}

void IdBatch::interp(const std::vector<double*>& P, const std::vector<int>& ldp, cudaStream_t s) {
  std::vector<IdProb> ip;
  int mx = 0;
  for (size_t id = 0; id < jobs.size(); ++id) {
    if (!P[id]) continue;
    const Job& j = jobs[id];
    IdProb q{};
    q.W = W.p + j.woff;
    q.ldw = j.nr;
    q.nr = j.nr;
    q.nc = j.spec.m;
    q.piv = piv.p + j.moff;
    q.norms = norms.p + j.noff;
    q.P = P[id];
    q.ldp = ldp[id];
    q.rank = rank.p + id;
    ip.push_back(q);
    mx = std::max(mx, j.spec.m * h_rank[id]);
  }
  batched_id_interp(ip, mx, s);
}

std::vector<int> IdBatch::pivots(cudaStream_t s) const { return piv.download(s); }

// ====================================================================== tree ID
// Largest level (number of problems) that is merged into a single root
// (RW_ROOT_MERGE overrides it, for tuning).
int root_merge_jobs() {
  static const int v = [] {
    const char* e = std::getenv("RW_ROOT_MERGE");
    const int x = e ? std::atoi(e) : 0;
    return x > 0 ? x : 256;
  }();
  return v;
}
namespace {
__global__ void k_gather_cols(const double* Z, int nr, const int* cand, int n, double* W) {
  for (int c = blockIdx.x; c < n; c += gridDim.x)
    for (int r = threadIdx.x; r < nr; r += blockDim.x) W[r + size_t(c) * nr] = Z[r + size_t(cand[c]) * nr];
}
}  // namespace

struct TreeId::Levels {
  // each job: candidate positions (into rows), indices of its child jobs in
  // the previous level, rank, skeleton positions, offset of its
  // interpolation matrix (m_j x k_j, ld m_j) in the level's buffer
  struct Job { std::vector<int> cand; std::vector<int> ch; int k = 0; std::vector<int> skel; size_t poff = 0; };
  std::vector<std::vector<Job>> levels;
  std::vector<DBuf<double>> Pl;
  int mt = 0;
};

DBuf<double> TreeId::expand(const double* T, int ldT, int kout, cudaStream_t s) const {
  if (!lv) {  // no rows at all
    require(k == 0, "TreeId::expand: no levels");
    return DBuf<double>(1);
  }
  if (!T) kout = k;
  const int mt = lv->mt;
  DBuf<double> out(std::max<size_t>(size_t(mt) * kout, 1));
  if (kout == 0) return out;
  if (k == 0) {
    fill_zero(out.p, size_t(mt) * kout, s);
    RW_CUDA(cudaStreamSynchronize(s));
    return out;
  }
  const auto& levels = lv->levels;
  const auto& Pl = lv->Pl;
  const auto& root = levels.back()[0];
  const int top = int(levels.size()) - 1;
  // the root's map of its candidates to the skeleton, times T
  auto root_map = [&](double* dst, int ld) {
    const int m = int(root.cand.size());
    if (T)
      batched_gemm({GemmProb{Pl[top].p + root.poff, T, dst, m, kout, k, m, ldT, ld, 0, 0, 1.0, 0.0}}, s);
    else
      RW_CUDA(cudaMemcpy2DAsync(dst, size_t(ld) * sizeof(double), Pl[top].p + root.poff, size_t(m) * sizeof(double),
                                size_t(m) * sizeof(double), size_t(k), cudaMemcpyDeviceToDevice, s));
  };
  if (top == 0) {
    root_map(out.p, mt);
    RW_CUDA(cudaStreamSynchronize(s));
    return out;
  }
  // top-down products: Wm[level][job] = (m_j x kout) map of candidates to
  // the root skeleton (times T)
  std::vector<DBuf<double>> Wm(levels.size());
  {
    size_t sz = 0;
    for (auto& j : levels[top]) sz += j.cand.size() * size_t(kout);
    Wm[top].alloc(std::max<size_t>(sz, 1));
    root_map(Wm[top].p, int(root.cand.size()));
  }
  for (int l = top; l > 0; --l) {
    auto& par = levels[l];
    auto& ch = levels[l - 1];
    std::vector<size_t> woff(ch.size());
    size_t sz = 0;
    for (size_t b = 0; b < ch.size(); ++b) { woff[b] = sz; sz += ch[b].cand.size() * size_t(kout); }
    const bool bottom = (l - 1 == 0);
    if (!bottom) Wm[l - 1].alloc(std::max<size_t>(sz, 1));
    std::vector<GemmProb> gm;
    std::vector<size_t> wpar(par.size());
    { size_t o = 0; for (size_t b = 0; b < par.size(); ++b) { wpar[b] = o; o += par[b].cand.size() * size_t(kout); } }
    for (size_t pb = 0; pb < par.size(); ++pb) {
      const int mp = int(par[pb].cand.size());
      int slice = 0;
      for (int cidx : par[pb].ch) {
        const auto& c = ch[cidx];
        const double* M = Wm[l].p + wpar[pb] + slice;  // rows slice of the parent's map, ld mp
        double* C;
        int ldc;
        if (bottom) { C = out.p + c.cand[0]; ldc = mt; } else { C = Wm[l - 1].p + woff[cidx]; ldc = int(c.cand.size()); }
        gm.push_back(GemmProb{Pl[l - 1].p + c.poff, M, C, int(c.cand.size()), kout, c.k, int(c.cand.size()), mp, ldc,
                              0, 0, 1.0, 0.0});
        slice += c.k;
      }
    }
    batched_gemm(gm, s);
  }
  // keep the temporaries alive until the stream has consumed them
  RW_CUDA(cudaStreamSynchronize(s));
  return out;
}

namespace {
TreeId tree_row_id_w(const NodesView& S, const std::vector<int>& rows, const IdMatProb& colspec,
                     const NodesView& E1, bool e1s, const NodesView& E2, bool e2s, double tol,
                     int sketch_cols, int sketch_width, unsigned long long seed, int chunk, cudaStream_t s,
                     bool defer);
}  // namespace

// Sketched problems first try a narrow sketch (kSketchTry rows) and keep it
// when the rank found leaves kSketchMargin rows of oversampling; otherwise
// they are redone at the full sketch width.
constexpr int kSketchTry = 96, kSketchMargin = 16;

TreeId tree_row_id(const NodesView& S, const std::vector<int>& rows, const IdMatProb& colspec,
                   const NodesView& E1, bool e1s, const NodesView& E2, bool e2s, double tol,
                   int sketch_cols, int sketch_width, unsigned long long seed, int chunk, cudaStream_t s,
                   bool defer) {
  const int ncol = idmat_ncol(0, colspec.n1, colspec.n2, idmat_nproxy(colspec), colspec.normal);
  if (ncol > sketch_cols && sketch_width > kSketchTry && ncol > kSketchTry) {
    TreeId t = tree_row_id_w(S, rows, colspec, E1, e1s, E2, e2s, tol, sketch_cols, kSketchTry, seed, chunk, s, defer);
    if (t.k <= kSketchTry - kSketchMargin) return t;
  }
  // A sketch of width w certifies ranks up to w - kSketchMargin only: a rank
  // beyond that means the sketch truncated the block, so the width doubles
  // until the rank leaves the margin or the sketch is no narrower than the
  // block itself (rows + margin, or every column).
  int w = sketch_width;
  for (;;) {
    TreeId t = tree_row_id_w(S, rows, colspec, E1, e1s, E2, e2s, tol, sketch_cols, w, seed, chunk, s, defer);
    const bool sketched = ncol > sketch_cols && w < ncol;
    if (!sketched || t.k <= w - kSketchMargin || w >= int(rows.size()) + kSketchMargin) return t;
    w = std::min(2 * w, std::max(int(rows.size()) + kSketchMargin, w + 1));
  }
}

namespace {
TreeId tree_row_id_w(const NodesView& S, const std::vector<int>& rows, const IdMatProb& colspec,
                     const NodesView& E1, bool e1s, const NodesView& E2, bool e2s, double tol,
                     int sketch_cols, int sketch_width, unsigned long long seed, int chunk, cudaStream_t s,
                     bool defer) {
  TreeId out;
  const int mt = int(rows.size());
  if (mt == 0) return out;
  Trace tr(s, "  tree-id");
  auto drows = to_device_tmp(rows, s);
  IdMatProb sp = colspec;
  sp.kind = 0;
  sp.m = mt;
  sp.cand = drows.p;
  sp.ncol = idmat_ncol(0, sp.n1, sp.n2, idmat_nproxy(sp), sp.normal);
  // Y^T for all rows, optionally sketched
  int nr = sp.ncol;
  TBuf<double> Yt(size_t(sp.ncol) * mt, s);
  sp.W = Yt.p;
  sp.ldw = sp.ncol;
  eval_idmat({sp}, S, E1, e1s, E2, e2s, s);
  TBuf<double> Zt;
  const double* Z = Yt.p;
  if (sp.ncol > sketch_cols && sketch_width < sp.ncol) {
    nr = sketch_width;
    TBuf<double> Om(size_t(sp.ncol) * nr, s);
    fill_rademacher(Om.p, Om.n, seed, s);
    Zt = TBuf<double>(size_t(nr) * mt, s);
    batched_gemm({GemmProb{Om.p, Yt.p, Zt.p, nr, mt, sp.ncol, sp.ncol, sp.ncol, nr, 1, 0, 1.0, 0.0}}, s);
    Z = Zt.p;
  }
  TBuf<double> mx(1, s);
  max_colnorm(Z, nr, mt, nr, mx.p, s);
  double hmx = 0;
  RW_CUDA(cudaMemcpyAsync(&hmx, mx.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  RW_CUDA(cudaStreamSynchronize(s));
  const double tol_abs = tol * hmx;
  tr.mark("eval (+sketch)");

  // level structure: each job has candidate positions (into rows) and the
  // indices of its child jobs in the previous level
  using TJob = TreeId::Levels::Job;
  out.lv = std::make_shared<TreeId::Levels>();
  out.lv->mt = mt;
  std::vector<std::vector<TJob>>& levels = out.lv->levels;
  std::vector<DBuf<double>>& Pl = out.lv->Pl;  // per level: interpolation matrices (m_j x k_j, ld m_j)
  std::vector<TJob> cur;
  if (const char* e = std::getenv("RW_TREE_CHUNK")) {
    const int x = std::atoi(e);
    if (x >= 16 && x <= 1024) chunk = x;
  }
  // a block of at most two chunks is one problem: a second level would add a
  // whole chain of pivot steps for no reduction in work
  if (mt <= 2 * chunk) chunk = mt;
  for (int r0 = 0; r0 < mt; r0 += chunk) {
    TJob j;
    for (int r = r0; r < std::min(mt, r0 + chunk); ++r) j.cand.push_back(r);
    cur.push_back(j);
  }
  while (true) {
    std::vector<int> cand_all;
    for (auto& j : cur) cand_all.insert(cand_all.end(), j.cand.begin(), j.cand.end());
    auto dcand = to_device_tmp(cand_all, s);
    TBuf<double> Wl(size_t(nr) * cand_all.size(), s);
    TBuf<double> nrm(2 * cand_all.size() + 4 * cur.size(), s);
    TBuf<int> piv(cand_all.size(), s), rk(cur.size(), s);
    k_gather_cols<<<std::min(ceil_div((long long)nr * cand_all.size(), 256), 4096), 256, 0, s>>>(
        Z, nr, dcand.p, int(cand_all.size()), Wl.p);
    RW_CHECK_LAUNCH();
    std::vector<IdProb> ip;
    size_t off = 0;
    for (size_t b = 0; b < cur.size(); ++b) {
      IdProb q{};
      q.W = Wl.p + off * nr;
      q.ldw = nr;
      q.nr = nr;
      q.nc = int(cur[b].cand.size());
      q.tol_abs = tol_abs;
      q.tol_rel = 0.0;
      q.min_rank = 0;
      q.max_rank = q.nc;
      q.piv = piv.p + off;
      q.norms = nrm.p + 2 * off + 4 * b;
      q.P = nullptr;
      q.ldp = q.nc;
      q.rank = rk.p + b;
      ip.push_back(q);
      off += cur[b].cand.size();
    }
    batched_id(ip, s);
    std::vector<int> hk(cur.size()), hp(cand_all.size());
    RW_CUDA(cudaMemcpyAsync(hk.data(), rk.p, hk.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    RW_CUDA(cudaMemcpyAsync(hp.data(), piv.p, hp.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    RW_CUDA(cudaStreamSynchronize(s));
    size_t psz = 0;
    off = 0;
    int mxe = 0;
    for (size_t b = 0; b < cur.size(); ++b) {
      cur[b].k = hk[b];
      cur[b].skel.clear();
      for (int i = 0; i < hk[b]; ++i) cur[b].skel.push_back(cur[b].cand[hp[off + i]]);
      cur[b].poff = psz;
      psz += cur[b].cand.size() * size_t(hk[b]);
      mxe = std::max(mxe, int(cur[b].cand.size()) * hk[b]);
      off += cur[b].cand.size();
    }
    DBuf<double> P(std::max<size_t>(psz, 1));
    for (size_t b = 0; b < cur.size(); ++b) {
      ip[b].P = P.p + cur[b].poff;
      ip[b].ldp = int(cur[b].cand.size());
    }
    batched_id_interp(ip, mxe, s);
    Pl.push_back(std::move(P));
    levels.push_back(cur);
    if (tr.on) {
      long long ksum = 0;
      int kmax = 0;
      for (auto& j : cur) { ksum += j.k; kmax = std::max(kmax, j.k); }
      char msg[160];
      std::snprintf(msg, sizeof msg, "%s: %zu problems, %d x %zu candidates, ranks sum %lld max %d",
                    cur.size() == 1 ? "level (root)" : "level", cur.size(), nr, cand_all.size(), ksum, kmax);
      tr.mark(msg);
    }
    if (cur.size() == 1) break;
    // Next level: pairwise merges while the level has enough problems to
    // occupy the GPU; once it has few, one root over every remaining
    // skeleton (one wide problem that the grid-wide factorisation spreads
    // over all SMs) replaces the remaining levels of narrow problems.
    size_t nsk = 0;
    for (auto& j : cur) nsk += j.skel.size();
    const bool wide_root = cur.size() > 2 && cur.size() <= size_t(root_merge_jobs()) && grid_id_fits(nr, int(nsk));
    std::vector<TJob> nxt;
    if (wide_root) {
      TJob j;
      for (size_t b = 0; b < cur.size(); ++b) {
        j.ch.push_back(int(b));
        j.cand.insert(j.cand.end(), cur[b].skel.begin(), cur[b].skel.end());
      }
      nxt.push_back(j);
    } else {
      for (size_t b = 0; b < cur.size(); b += 2) {
        TJob j;
        j.ch.push_back(int(b));
        j.cand = cur[b].skel;
        if (b + 1 < cur.size()) {
          j.ch.push_back(int(b + 1));
          j.cand.insert(j.cand.end(), cur[b + 1].skel.begin(), cur[b + 1].skel.end());
        }
        nxt.push_back(j);
      }
    }
    // keep the (small) sync-free guard: wait for this level's buffers before reuse
    cur = nxt;
  }
  const TJob& root = levels.back()[0];
  out.k = root.k;
  out.skel = root.skel;
  RW_CUDA(cudaStreamSynchronize(s));  // the levels are complete (a deferred expansion may use another stream)
  if (defer) return out;
  out.P = out.expand(nullptr, 0, 0, s);
  tr.mark("top-down interpolation");
  return out;
}
}  // namespace

// ====================================================================== HBS build
namespace {

struct Geo { double cx, cy, rad; };

Geo node_geo(const std::vector<double>& x, const std::vector<double>& y, int lo, int hi) {
  double cx = 0, cy = 0;
  for (int i = lo; i < hi; ++i) { cx += x[i]; cy += y[i]; }
  cx /= (hi - lo);
  cy /= (hi - lo);
  double r2 = 0;
  for (int i = lo; i < hi; ++i) r2 = std::max(r2, (x[i] - cx) * (x[i] - cx) + (y[i] - cy) * (y[i] - cy));
  return Geo{cx, cy, std::sqrt(r2)};
}

}  // namespace

void Hbs::build(const Nodes& nodes, const Opts& o, cudaStream_t s, bool fwd_only) {
  Trace tr(s, "hbs");
  N = nodes.n;
  require(N >= 1, "HBS: empty node set");
  L = 0;
  while ((N + (1 << L) - 1) / (1 << L) > o.leaf_points) ++L;
  node.assign(size_t(2) << L, HbsNode());
  node[1].lo = 0;
  node[1].hi = N;
  for (int h = 1; h < (1 << L); ++h) {
    const int mid = (node[h].lo + node[h].hi) / 2;
    node[2 * h].lo = node[h].lo;
    node[2 * h].hi = mid;
    node[2 * h + 1].lo = mid;
    node[2 * h + 1].hi = node[h].hi;
  }
  lev.clear();
  lev.resize(L + 1);
  const NodesView V = nodes.view();
  const auto& hx = nodes.hx;
  const auto& hy = nodes.hy;
  max_rank = 0;
  bytes = 0;

  // ---------------------------------------------------------- leaf D blocks
  {
    Level& LL = lev[L];
    const int nl = 1 << L;
    LL.oD.resize(nl);
    size_t sd = 0;
    for (int t = 0; t < nl; ++t) { const HbsNode& nd = node[nl + t]; LL.oD[t] = sd; sd += size_t(4) * (nd.hi - nd.lo) * (nd.hi - nd.lo); }
    LL.D.alloc(sd);
    std::vector<BlockProb> bp;
    for (int t = 0; t < nl; ++t) {
      const HbsNode& nd = node[nl + t];
      const int n = 2 * (nd.hi - nd.lo);
      bp.push_back(BlockProb{n, n, nullptr, nullptr, 2 * nd.lo, 2 * nd.lo, 0, 0, 1.0, LL.D.p + LL.oD[t], n});
    }
    eval_blocks(bp, V, V, s);
  }
  // ---------------------------------------------------------- inverse (pipelined)
  // Per node: D~ (leaf: D; parent: [Dh_a B12; B21 Dh_b]); Dinv = D~^{-1};
  // Dh = (V* Dinv U)^{-1}; E = Dinv U Dh; F* = Dh V* Dinv; G = Dinv - E V* Dinv.
  // Level l needs its own U, V* (compression of level l), its B blocks (the
  // skeletons of level l + 1) and the children's Dh (inverse of level l + 1):
  // it runs on its own stream as soon as level l is compressed, while the
  // host goes on compressing level l - 1.  Buffers that outlive the build are
  // allocated on the build's stream and handed over through an event; the
  // inverse's temporaries (the children's Dh included) live on its stream.
  // declaration order = reverse destruction order: on any exit the inverse
  // stream is synchronised (done) after its own temporaries are released and
  // before anything it reads (flags, index lists) is
  DBuf<int> flags(size_t(2) << L);
  flags.zero(s);
  std::vector<DBuf<int>> keep_idx;  // B-block index lists, alive until the inverse stream is done
  cudaStream_t si = nullptr;
  cudaEvent_t ev_alloc = nullptr;
  struct StreamDone {
    cudaStream_t& st;
    cudaEvent_t& ev;
    ~StreamDone() {
      if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
      if (ev) cudaEventDestroy(ev);
    }
  } done{si, ev_alloc};
  RW_CUDA(cudaStreamCreateWithFlags(&si, cudaStreamNonBlocking));
  RW_CUDA(cudaEventCreateWithFlags(&ev_alloc, cudaEventDisableTiming));
  TBuf<double> Dh_prev;  // Dh of the level below (children), offsets koff^2, on si
  std::vector<size_t> oDh_prev;
  auto order_after_alloc = [&] {
    RW_CUDA(cudaEventRecord(ev_alloc, s));
    RW_CUDA(cudaStreamWaitEvent(si, ev_alloc, 0));
  };
  auto invert_level = [&](int l) {
    const int h0 = 1 << l, nn = 1 << l;
    Level& LV = lev[l];
    if (l < L) {
      // B blocks between the children of every node of level l
      LV.oB12.resize(nn); LV.oB21.resize(nn);
      size_t sb = 0;
      std::vector<int> idx;
      std::vector<size_t> pos;
      for (int t = 0; t < nn; ++t) {
        const HbsNode& a = node[2 * (h0 + t)];
        const HbsNode& b = node[2 * (h0 + t) + 1];
        LV.oB12[t] = sb; sb += size_t(a.k) * b.k;
        LV.oB21[t] = sb; sb += size_t(b.k) * a.k;
        for (const std::vector<int>* v : {&a.skr, &b.skc, &b.skr, &a.skc}) { pos.push_back(idx.size()); idx.insert(idx.end(), v->begin(), v->end()); }
      }
      LV.B.alloc(std::max<size_t>(sb, 1));
      keep_idx.push_back(to_device(idx, s));
      order_after_alloc();
      const int* di = keep_idx.back().p;
      std::vector<BlockProb> bp;
      for (int t = 0; t < nn; ++t) {
        const HbsNode& a = node[2 * (h0 + t)];
        const HbsNode& b = node[2 * (h0 + t) + 1];
        bp.push_back(BlockProb{a.k, b.k, di + pos[4 * t], di + pos[4 * t + 1], 0, 0, 0, 0, 1.0, LV.B.p + LV.oB12[t], a.k});
        bp.push_back(BlockProb{b.k, a.k, di + pos[4 * t + 2], di + pos[4 * t + 3], 0, 0, 0, 0, 1.0, LV.B.p + LV.oB21[t], b.k});
      }
      eval_blocks(bp, V, V, si);
    } else {
      order_after_alloc();  // the leaf D blocks and this level's U, V*
    }
    if (fwd_only) return;
    std::vector<int> mm(nn);
    size_t sG = 0;
    LV.oG.resize(nn);
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      mm[t] = (l == L) ? 2 * (nd.hi - nd.lo) : node[2 * (h0 + t)].k + node[2 * (h0 + t) + 1].k;
      if (l > 0) require(mm[t] == nd.m, "HBS: inconsistent candidate count");
      LV.oG[t] = sG;
      sG += size_t(mm[t]) * mm[t];
    }
    LV.G.alloc(sG);
    order_after_alloc();
    TBuf<double> Dt(sG, si), Wk(sG, si);
    // assemble D~
    std::vector<CopyProb> cp;
    for (int t = 0; t < nn; ++t) {
      const int n = mm[t];
      double* dst = Dt.p + LV.oG[t];
      if (l == L) {
        cp.push_back(CopyProb{LV.D.p + LV.oD[t], n, n, n, dst, n});
      } else {
        const HbsNode& a = node[2 * (h0 + t)];
        const HbsNode& b = node[2 * (h0 + t) + 1];
        const int ca = 2 * t, cb = 2 * t + 1;  // child positions in the level below
        cp.push_back(CopyProb{Dh_prev.p + oDh_prev[ca], a.k, a.k, a.k, dst, n});
        cp.push_back(CopyProb{Dh_prev.p + oDh_prev[cb], b.k, b.k, b.k, dst + a.k + size_t(a.k) * n, n});
        cp.push_back(CopyProb{LV.B.p + LV.oB12[t], a.k, b.k, a.k, dst + size_t(a.k) * n, n});
        cp.push_back(CopyProb{LV.B.p + LV.oB21[t], b.k, a.k, b.k, dst + a.k, n});
      }
    }
    batched_copy(cp, si);
    // Dinv into G (root: final)
    std::vector<InvProb> inv;
    for (int t = 0; t < nn; ++t)
      inv.push_back(InvProb{Dt.p + LV.oG[t], LV.G.p + LV.oG[t], Wk.p + LV.oG[t], mm[t], mm[t], mm[t], flags.p + h0 + t});
    batched_inverse(inv, si);
    if (l == 0) return;
    // T1 = Dinv U (m x k), T2 = Vt Dinv (k x m), M = Vt T1 (k x k)
    size_t sk = 0, skk = 0;
    std::vector<size_t> oT(nn), oK(nn);
    for (int t = 0; t < nn; ++t) { oT[t] = sk; sk += size_t(mm[t]) * node[h0 + t].k; oK[t] = skk; skk += size_t(node[h0 + t].k) * node[h0 + t].k; }
    LV.E.alloc(sk); LV.F.alloc(sk);
    order_after_alloc();
    TBuf<double> T1(sk, si), T2(sk, si), M(skk, si), Mw(skk, si);
    TBuf<double> Dh(std::max<size_t>(skk, 1), si);
    LV.oE = oT; LV.oF = oT;
    std::vector<GemmProb> g1, g2;
    for (int t = 0; t < nn; ++t) {
      const int n = mm[t], k = node[h0 + t].k;
      const double* Di = LV.G.p + LV.oG[t];
      g1.push_back(GemmProb{Di, LV.U.p + LV.oU[t], T1.p + oT[t], n, k, n, n, n, n, 0, 0, 1.0, 0.0});
      g1.push_back(GemmProb{LV.Vt.p + LV.oVt[t], Di, T2.p + oT[t], k, n, n, k, n, k, 0, 0, 1.0, 0.0});
    }
    batched_gemm(g1, si);
    for (int t = 0; t < nn; ++t) {
      const int n = mm[t], k = node[h0 + t].k;
      g2.push_back(GemmProb{LV.Vt.p + LV.oVt[t], T1.p + oT[t], M.p + oK[t], k, k, n, k, n, k, 0, 0, 1.0, 0.0});
    }
    batched_gemm(g2, si);
    std::vector<InvProb> inv2;
    for (int t = 0; t < nn; ++t)
      inv2.push_back(InvProb{M.p + oK[t], Dh.p + oK[t], Mw.p + oK[t], node[h0 + t].k, node[h0 + t].k, node[h0 + t].k, flags.p + h0 + t});
    batched_inverse(inv2, si);
    std::vector<GemmProb> g3, g4;
    for (int t = 0; t < nn; ++t) {
      const int n = mm[t], k = node[h0 + t].k;
      g3.push_back(GemmProb{T1.p + oT[t], Dh.p + oK[t], LV.E.p + oT[t], n, k, k, n, k, n, 0, 0, 1.0, 0.0});
      g3.push_back(GemmProb{Dh.p + oK[t], T2.p + oT[t], LV.F.p + oT[t], k, n, k, k, k, k, 0, 0, 1.0, 0.0});
    }
    batched_gemm(g3, si);
    for (int t = 0; t < nn; ++t) {
      const int n = mm[t], k = node[h0 + t].k;
      g4.push_back(GemmProb{LV.E.p + oT[t], T2.p + oT[t], LV.G.p + LV.oG[t], n, n, k, n, k, n, 0, 0, -1.0, 1.0});
    }
    batched_gemm(g4, si);
    Dh_prev = std::move(Dh);
    oDh_prev = oK;
  };
  // ---------------------------------------------------------- compression
  // Exterior walls: besides the points inside a node's proxy circle, every
  // point of a panel that shares a singular-rule pair with one of the node's
  // panels is taken explicitly (its entries are not the smooth kernel's)
  const bool ext = nodes.kind == kNodesExterior;
  std::vector<std::vector<int>> ext_nb;
  if (ext) ext_nb = ext_panel_neighbours(nodes);
  for (int l = L; l >= 1; --l) {
    const int h0 = 1 << l, nn = 1 << l;
    std::vector<int> idx;  // candidate / near index lists, concatenated
    std::vector<size_t> o_cr(nn), o_cc(nn), o_near(nn);
    std::vector<int> n_near(nn), m(nn);
    std::vector<Geo> geo(nn);
    for (int t = 0; t < nn; ++t) {
      HbsNode& nd = node[h0 + t];
      std::vector<int> cr, cc;
      if (l == L) {
        for (int d = 2 * nd.lo; d < 2 * nd.hi; ++d) cr.push_back(d);
        cc = cr;
      } else {
        const HbsNode& a = node[2 * (h0 + t)];
        const HbsNode& b = node[2 * (h0 + t) + 1];
        cr = a.skr; cr.insert(cr.end(), b.skr.begin(), b.skr.end());
        cc = a.skc; cc.insert(cc.end(), b.skc.begin(), b.skc.end());
      }
      nd.m = int(cr.size());
      m[t] = nd.m;
      geo[t] = node_geo(hx, hy, nd.lo, nd.hi);
      const double R = o.proxy_ratio * geo[t].rad, R2 = R * R;
      o_cr[t] = idx.size(); idx.insert(idx.end(), cr.begin(), cr.end());
      o_cc[t] = idx.size(); idx.insert(idx.end(), cc.begin(), cc.end());
      o_near[t] = idx.size();
      int cnt = 0;
      for (int j = 0; j < N; ++j) {
        if (j >= nd.lo && j < nd.hi) continue;
        const double dx = hx[j] - geo[t].cx, dy = hy[j] - geo[t].cy;
        if (dx * dx + dy * dy < R2) { idx.push_back(2 * j); idx.push_back(2 * j + 1); cnt += 2; }
      }
      if (ext) {
        std::vector<int> extra;
        for (int p = nd.lo / 16; p <= (nd.hi - 1) / 16; ++p)
          for (int qn : ext_nb[p])
            for (int j = 16 * qn; j < 16 * qn + 16; ++j) {
              if (j >= nd.lo && j < nd.hi) continue;
              const double dx = hx[j] - geo[t].cx, dy = hy[j] - geo[t].cy;
              if (dx * dx + dy * dy >= R2) extra.push_back(j);
            }
        std::sort(extra.begin(), extra.end());
        extra.erase(std::unique(extra.begin(), extra.end()), extra.end());
        for (int j : extra) { idx.push_back(2 * j); idx.push_back(2 * j + 1); cnt += 2; }
      }
      n_near[t] = cnt;
    }
    DBuf<int> didx = to_device(idx, s);
    IdBatch batch;
    batch.paired = true;
    for (int t = 0; t < nn; ++t) {
      const double R = o.proxy_ratio * geo[t].rad;
      for (int kind = 0; kind < 2; ++kind) {
        IdMatProb p{};
        p.kind = kind;
        p.m = m[t];
        p.cand = didx.p + (kind == 0 ? o_cr[t] : o_cc[t]);
        p.n1 = n_near[t];
        p.e1 = didx.p + o_near[t];
        p.n2 = 0;
        p.e2 = nullptr;
        p.cx = geo[t].cx;
        p.cy = geo[t].cy;
        p.R = R;
        p.M = o.n_proxy;
        p.normal = ext ? 0 : 1;            // the exterior operator has no N term
        p.sl_in = (ext && kind == 1) ? 1 : 0;  // sources carry the combined field
        batch.add(p, o.sketch_cols, m[t] + 16);
      }
    }
    batch.run(V, V, true, V, true, o.id_tol, {}, {}, {}, {}, o.seed + l, s);
    if (tr.on) {
      long long msum = 0, ksum = 0;
      int kmax = 0;
      for (int t = 0; t < nn; ++t) msum += m[t];
      for (int j = 0; j < 2 * nn; ++j) { ksum += batch.h_rank[j]; kmax = std::max(kmax, batch.h_rank[j]); }
      char msg[160];
      std::snprintf(msg, sizeof msg, "  level %d IDs: %d nodes, candidates %lld, feature rows %d..%d, ranks sum %lld max %d",
                    l, nn, msum, batch.jobs.front().nr, batch.jobs.back().nr, ksum, kmax);
      tr.mark(msg);
    }
    std::vector<int> kfix(2 * nn), redo, minr(2 * nn, 0), maxr(2 * nn);
    for (int t = 0; t < nn; ++t) {
      int k = std::max(batch.h_rank[2 * t], batch.h_rank[2 * t + 1]);
      k = std::max(1, std::min(k, m[t]));
      node[h0 + t].k = k;
      for (int q = 0; q < 2; ++q) {
        maxr[2 * t + q] = k;
        minr[2 * t + q] = k;
        if (batch.h_rank[2 * t + q] != k) redo.push_back(2 * t + q);
      }
    }
    if (!redo.empty()) batch.run(V, V, true, V, true, 0.0, {}, redo, minr, maxr, o.seed + l, s);
    tr.mark("  level IDs at the common rank");
    // storage for U (m x k), V (m x k -> transposed to Vt)
    Level& LV = lev[l];
    LV.oU.resize(nn); LV.oVt.resize(nn);
    LV.koff.assign(nn + 1, 0);
    size_t su = 0;
    for (int t = 0; t < nn; ++t) {
      LV.oU[t] = su;
      su += size_t(m[t]) * node[h0 + t].k;
      LV.koff[t + 1] = LV.koff[t] + node[h0 + t].k;
      max_rank = std::max(max_rank, node[h0 + t].k);
    }
    LV.oVt = LV.oU;
    LV.U.alloc(std::max<size_t>(su, 1));
    LV.Vt.alloc(std::max<size_t>(su, 1));
    TBuf<double> Vtmp(std::max<size_t>(su, 1), s);
    std::vector<double*> Pp(2 * nn);
    std::vector<int> ldp(2 * nn);
    for (int t = 0; t < nn; ++t) {
      Pp[2 * t] = LV.U.p + LV.oU[t]; ldp[2 * t] = m[t];
      Pp[2 * t + 1] = Vtmp.p + LV.oU[t]; ldp[2 * t + 1] = m[t];
    }
    batch.interp(Pp, ldp, s);
    std::vector<TransProb> tp;
    for (int t = 0; t < nn; ++t) tp.push_back(TransProb{Vtmp.p + LV.oU[t], m[t], node[h0 + t].k, m[t], LV.Vt.p + LV.oVt[t], node[h0 + t].k});
    batched_transpose(tp, s);
    auto piv = batch.pivots(s);
    for (int t = 0; t < nn; ++t) {
      HbsNode& nd = node[h0 + t];
      nd.skr.resize(nd.k);
      nd.skc.resize(nd.k);
      for (int i = 0; i < nd.k; ++i) {
        nd.skr[i] = idx[o_cr[t] + piv[batch.piv_off(2 * t) + i]];
        nd.skc[i] = idx[o_cc[t] + piv[batch.piv_off(2 * t + 1) + i]];
      }
    }
    RW_CUDA(cudaStreamSynchronize(s));
    invert_level(l);
  }

  tr.mark("compression (IDs), inverse overlapped");
  invert_level(0);
  Dh_prev = TBuf<double>();
  RW_CUDA(cudaStreamSynchronize(si));
  auto hf = flags.download(s);
  for (int f : hf) require(f == 0, "HBS inverse: singular diagonal block", RW_ERR_SINGULAR);

  tr.mark("inverse");
  // ---------------------------------------------------------- statistics
  inv_elems = fwd_elems = 0;
  bytes = 0;
  for (int l = 0; l <= L; ++l) {
    Level& LV = lev[l];
    inv_elems += (long long)LV.G.n + (l > 0 ? (long long)LV.E.n + (long long)LV.F.n : 0);
    fwd_elems += (long long)LV.U.n * (l > 0) + (long long)LV.Vt.n * (l > 0) + (long long)LV.B.n * (l < L) + (long long)LV.D.n;
    bytes += LV.U.bytes() + LV.Vt.bytes() + LV.E.bytes() + LV.F.bytes() + LV.G.bytes() + LV.B.bytes() + LV.D.bytes();
  }
}

// dense single-leaf inverses above this size use block Gauss-Jordan with
// diagonal blocks of kBlockInverseNb rows (each inverted in shared memory)
constexpr int kBlockInverseMin = 512, kBlockInverseNb = 320;

void Hbs::build_dense(DBuf<double>&& A, int npts, cudaStream_t s) {
  N = npts;
  require(N >= 1, "HBS: empty node set");
  const int n = 2 * N;
  require(A.n >= size_t(n) * n, "HBS: dense matrix too small");
  L = 0;
  node.assign(2, HbsNode());
  node[1].lo = 0;
  node[1].hi = N;
  lev.clear();
  lev.resize(1);
  Level& LV = lev[0];
  LV.D = std::move(A);
  LV.oD = {0};
  LV.oG = {0};
  LV.G.alloc(size_t(n) * n);
  DBuf<int> flag(1);
  flag.zero(s);
  if (n > kBlockInverseMin) {
    // beyond one shared-memory cluster: block Gauss-Jordan on GEMMs
    block_inverse(LV.D.p, LV.G.p, n, kBlockInverseNb, flag.p, s);
  } else {
    TBuf<double> Dt(size_t(n) * n, s), Wk(size_t(n) * n, s);
    batched_copy({CopyProb{LV.D.p, n, n, n, Dt.p, n}}, s);
    batched_inverse({InvProb{Dt.p, LV.G.p, Wk.p, n, n, n, flag.p}}, s);
  }
  const auto hf = flag.download(s);
  require(hf[0] == 0, "HBS inverse: singular dense block", RW_ERR_SINGULAR);
  max_rank = 0;
  inv_elems = (long long)LV.G.n;
  fwd_elems = (long long)LV.D.n;
  bytes = LV.G.bytes() + LV.D.bytes();
}

void Hbs::make_bf16(cudaStream_t s) {
  for (int l = 0; l <= L; ++l) {
    Level& LV = lev[l];
    LV.G16.alloc(LV.G.n); copy_d2bf(LV.G.p, LV.G16.p, LV.G.n, s);
    if (l > 0) {
      LV.E16.alloc(LV.E.n); copy_d2bf(LV.E.p, LV.E16.p, LV.E.n, s);
      LV.F16.alloc(LV.F.n); copy_d2bf(LV.F.p, LV.F16.p, LV.F.n, s);
    }
  }
  has_bf16 = true;
}

void Hbs::make_fp32(cudaStream_t s) {
  for (int l = 0; l <= L; ++l) {
    Level& LV = lev[l];
    LV.G32.alloc(LV.G.n); copy_d2f(LV.G.p, LV.G32.p, LV.G.n, s);
    if (l > 0) {
      LV.E32.alloc(LV.E.n); copy_d2f(LV.E.p, LV.E32.p, LV.E.n, s);
      LV.F32.alloc(LV.F.n); copy_d2f(LV.F.p, LV.F32.p, LV.F.n, s);
    }
  }
  has_fp32 = true;
}

// ====================================================================== sweeps
template <class T, class MT>
void Hbs::sweep_inverse(const T* b, T* x, int nrhs, cudaStream_t s) const {
  const int ld = 2 * N;
  // matrices in MT: the FP64 factors, or their FP32 / BF16 copies
  auto pick = [](const DBuf<double>& d, const DBuf<float>& f, const DBuf<__nv_bfloat16>& h) -> const MT* {
    if constexpr (std::is_same<MT, double>::value) return d.p;
    else if constexpr (std::is_same<MT, float>::value) return f.p;
    else return h.p;
  };
  // many right-hand sides: the cached GEMM program (one launch per 64)
  if (nrhs > 8) {
    if constexpr (std::is_same<T, double>::value) inverse_gemm(b, x, nrhs, s);
    else inverse_gemm_f32(b, x, nrhs, std::is_same<MT, __nv_bfloat16>::value, s);
    return;
  }
  auto Gp = [&](const Level& LV) -> const MT* { return pick(LV.G, LV.G32, LV.G16); };
  auto Ep = [&](const Level& LV) -> const MT* { return pick(LV.E, LV.E32, LV.E16); };
  auto Fp = [&](const Level& LV) -> const MT* { return pick(LV.F, LV.F32, LV.F16); };
  if (L == 0) {
    matvec<T, MT>({GemvProb<T, MT>{Gp(lev[0]), b, x, ld, ld, ld, ld, ld, 1.0, 0.0}}, nrhs, s);
    return;
  }
  // per-level vectors uh (K_l x nrhs) and qh (K_l x nrhs)
  std::vector<TBuf<T>> uh(L + 1), qh(L + 1);
  for (int l = 1; l <= L; ++l) {
    const int K = lev[l].koff.back();
    uh[l] = TBuf<T>(size_t(K) * nrhs, s);
    qh[l] = TBuf<T>(size_t(K) * nrhs, s);
  }
  // up: leaves
  {
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const int K = LV.koff.back();
    std::vector<GemvProb<T, MT>> ps;
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo), k = nd.k;
      const T* in = b + 2 * nd.lo;
      ps.push_back(GemvProb<T, MT>{Fp(LV) + LV.oF[t], in, uh[l].p + LV.koff[t], k, n, k, ld, K, 1.0, 0.0});
      ps.push_back(GemvProb<T, MT>{Gp(LV) + LV.oG[t], in, x + 2 * nd.lo, n, n, n, ld, ld, 1.0, 0.0});
    }
    matvec<T, MT>(ps, nrhs, s);
  }
  for (int l = L - 1; l >= 1; --l) {
    const int h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    const int K = LV.koff.back(), KC = LC.koff.back();
    std::vector<GemvProb<T, MT>> ps;
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = nd.m, k = nd.k;
      const T* in = uh[l + 1].p + LC.koff[2 * t];
      ps.push_back(GemvProb<T, MT>{Fp(LV) + LV.oF[t], in, uh[l].p + LV.koff[t], k, n, k, KC, K, 1.0, 0.0});
      ps.push_back(GemvProb<T, MT>{Gp(LV) + LV.oG[t], in, qh[l + 1].p + LC.koff[2 * t], n, n, n, KC, KC, 1.0, 0.0});
    }
    matvec<T, MT>(ps, nrhs, s);
  }
  {
    const int K1 = lev[1].koff.back();
    matvec<T, MT>({GemvProb<T, MT>{Gp(lev[0]), uh[1].p, qh[1].p, K1, K1, K1, K1, K1, 1.0, 0.0}}, nrhs, s);
  }
  for (int l = 1; l <= L - 1; ++l) {
    const int h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    const int K = LV.koff.back(), KC = LC.koff.back();
    std::vector<GemvProb<T, MT>> ps;
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      ps.push_back(GemvProb<T, MT>{Ep(LV) + LV.oE[t], qh[l].p + LV.koff[t], qh[l + 1].p + LC.koff[2 * t], nd.m, nd.k, nd.m, K, KC, 1.0, 1.0});
    }
    matvec<T, MT>(ps, nrhs, s);
  }
  {
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const int K = LV.koff.back();
    std::vector<GemvProb<T, MT>> ps;
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      ps.push_back(GemvProb<T, MT>{Ep(LV) + LV.oE[t], qh[l].p + LV.koff[t], x + 2 * nd.lo, n, nd.k, n, K, ld, 1.0, 1.0});
    }
    matvec<T, MT>(ps, nrhs, s);
  }
}

void Hbs::apply_inverse(const double* b, double* x, int nrhs, cudaStream_t s) const {
  if (nrhs <= 8) apply_inverse_program(b, x, nrhs, s);
  else sweep_inverse<double, double>(b, x, nrhs, s);
}

int Hbs::emit_inverse_sweep(Program& P, int p0, int in_b, long long in_o, int in_ld, int out_b, long long out_o,
                            int out_ld) const {
  constexpr int WS = 2;  // workspace base
  if (L == 0) {
    P.gemv(p0, lev[0].G.p, 2 * N, 2 * N, 2 * N, in_b, in_o, in_ld, out_b, out_o, out_ld, 1.0, 0.0);
    return p0 + 1;
  }
  std::vector<long long> uh(L + 1), qh(L + 1);
  for (int l = 1; l <= L; ++l) {
    uh[l] = P.ws_alloc(lev[l].koff.back());
    qh[l] = P.ws_alloc(lev[l].koff.back());
  }
  int p = p0;
  {  // leaves: u^ = F* u, x = G u
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      P.gemv(p, LV.F.p + LV.oF[t], nd.k, n, nd.k, in_b, in_o + 2 * nd.lo, in_ld, WS, uh[l] + LV.koff[t], -1, 1.0, 0.0);
      P.gemv(p, LV.G.p + LV.oG[t], n, n, n, in_b, in_o + 2 * nd.lo, in_ld, out_b, out_o + 2 * nd.lo, out_ld, 1.0, 0.0);
    }
    ++p;
  }
  for (int l = L - 1; l >= 1; --l, ++p) {
    const int h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const long long in = uh[l + 1] + LC.koff[2 * t];
      P.gemv(p, LV.F.p + LV.oF[t], nd.k, nd.m, nd.k, WS, in, -1, WS, uh[l] + LV.koff[t], -1, 1.0, 0.0);
      P.gemv(p, LV.G.p + LV.oG[t], nd.m, nd.m, nd.m, WS, in, -1, WS, qh[l + 1] + LC.koff[2 * t], -1, 1.0, 0.0);
    }
  }
  {
    const int K1 = lev[1].koff.back();
    P.gemv(p++, lev[0].G.p, K1, K1, K1, WS, uh[1], -1, WS, qh[1], -1, 1.0, 0.0);
  }
  for (int l = 1; l <= L - 1; ++l, ++p) {
    const int h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      P.gemv(p, LV.E.p + LV.oE[t], nd.m, nd.k, nd.m, WS, qh[l] + LV.koff[t], -1, WS, qh[l + 1] + LC.koff[2 * t], -1,
             1.0, 1.0);
    }
  }
  {
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      P.gemv(p, LV.E.p + LV.oE[t], n, nd.k, n, WS, qh[l] + LV.koff[t], -1, out_b, out_o + 2 * nd.lo, out_ld, 1.0, 1.0);
    }
    ++p;
  }
  return p;
}

int Hbs::emit_forward_sweep(Program& P, int p0, int in_b, long long in_o, int in_ld, int out_b, long long out_o,
                            int out_ld) const {
  constexpr int WS = 2;  // workspace base
  if (L == 0) {
    P.gemv(p0, lev[0].D.p, 2 * N, 2 * N, 2 * N, in_b, in_o, in_ld, out_b, out_o, out_ld, 1.0, 0.0);
    return p0 + 1;
  }
  std::vector<long long> xh(L + 1), yh(L + 1);
  for (int l = 1; l <= L; ++l) {
    xh[l] = P.ws_alloc(lev[l].koff.back());
    yh[l] = P.ws_alloc(lev[l].koff.back());
  }
  {  // leaves: x^ = V* x, y = D x
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      P.gemv(p0, LV.Vt.p + LV.oVt[t], nd.k, n, nd.k, in_b, in_o + 2 * nd.lo, in_ld, WS, xh[l] + LV.koff[t], -1, 1.0,
             0.0);
      P.gemv(p0, LV.D.p + LV.oD[t], n, n, n, in_b, in_o + 2 * nd.lo, in_ld, out_b, out_o + 2 * nd.lo, out_ld, 1.0, 0.0);
    }
  }
  for (int l = L - 1; l >= 0; --l) {  // up: x^_l = V* x^_{l+1}; siblings: y^ = B x^
    const int p = p0 + (L - l), h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      if (l >= 1)
        P.gemv(p, LV.Vt.p + LV.oVt[t], nd.k, nd.m, nd.k, WS, xh[l + 1] + LC.koff[2 * t], -1, WS, xh[l] + LV.koff[t], -1,
               1.0, 0.0);
      const HbsNode& a = node[2 * (h0 + t)];
      const HbsNode& b = node[2 * (h0 + t) + 1];
      const long long ia = LC.koff[2 * t], ib = LC.koff[2 * t + 1];
      P.gemv(p, LV.B.p + LV.oB12[t], a.k, b.k, a.k, WS, xh[l + 1] + ib, -1, WS, yh[l + 1] + ia, -1, 1.0, 0.0);
      P.gemv(p, LV.B.p + LV.oB21[t], b.k, a.k, b.k, WS, xh[l + 1] + ia, -1, WS, yh[l + 1] + ib, -1, 1.0, 0.0);
    }
  }
  for (int l = 1; l <= L - 1; ++l) {  // down: y^_{l+1} += U y^_l
    const int p = p0 + L + l, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      P.gemv(p, LV.U.p + LV.oU[t], nd.m, nd.k, nd.m, WS, yh[l] + LV.koff[t], -1, WS, yh[l + 1] + LC.koff[2 * t], -1,
             1.0, 1.0);
    }
  }
  {  // leaves: y += U y^
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      P.gemv(p0 + 2 * L, LV.U.p + LV.oU[t], n, nd.k, n, WS, yh[l] + LV.koff[t], -1, out_b, out_o + 2 * nd.lo, out_ld, 1.0,
             1.0);
    }
  }
  return p0 + 2 * L + 1;
}

void Hbs::apply_inverse_program(const double* b, double* x, int nrhs, cudaStream_t s) const {
  if (!inv_prog_built) {
    emit_inverse_sweep(inv_prog, 0, 0, 0, 2 * N, 1, 0, 2 * N);
    inv_prog.finalize(s);
    inv_prog_built = true;
  }
  const size_t need = size_t(std::max<long long>(inv_prog.ws_per_rhs(), 1)) * nrhs;
  if (prog_ws.n < need) prog_ws.alloc(need);
  double* bases[kMaxBases] = {const_cast<double*>(b), x, prog_ws.p, nullptr};
  inv_prog.run(bases, nrhs, s);
}
void Hbs::apply_inverse_f32(const float* b, float* x, int nrhs, cudaStream_t s) const {
  require(has_fp32, "HBS: FP32 copies not built");
  sweep_inverse<float, float>(b, x, nrhs, s);
}

void Hbs::apply_inverse_bf16(const float* b, float* x, int nrhs, cudaStream_t s) const {
  require(has_bf16, "HBS: BF16 copies not built");
  sweep_inverse<float, __nv_bfloat16>(b, x, nrhs, s);
}

void Hbs::apply_forward(const double* xin, double* y, int nrhs, cudaStream_t s) const {
  if (nrhs > 8) forward_gemm(xin, y, nrhs, false, s);
  else forward_impl<double>(xin, y, nrhs, s);
}

void Hbs::apply_forward_df(const double* xin, double* y, int nrhs, cudaStream_t s) const {
  make_df(s);
  if (nrhs > 8) forward_gemm(xin, y, nrhs, true, s);
  else forward_impl<float2>(xin, y, nrhs, s);
}

void Hbs::make_df(cudaStream_t s_caller) const {
  // once per representation; the wall's copy may be asked for by several
  // host threads (serving workers) at the same time
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (has_df) return;
  AllocStreamScope scope(own_stream);
  cudaStream_t s = own_stream ? own_stream : s_caller;  // copies ordered after the allocation
  for (int l = 0; l <= L; ++l) {
    const Level& LV = lev[l];
    for (auto pr : {std::make_pair(&LV.U, &LV.U2), std::make_pair(&LV.Vt, &LV.Vt2), std::make_pair(&LV.B, &LV.B2),
                    std::make_pair(&LV.D, &LV.D2)}) {
      pr.second->alloc(pr.first->n);
      copy_d2df(pr.first->p, pr.second->p, pr.first->n, s);
    }
  }
  RW_CUDA(cudaStreamSynchronize(s));
  has_df = true;
}

void Hbs::make_df_inv(cudaStream_t s_caller) const {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (has_df_inv) return;
  AllocStreamScope scope(own_stream);
  cudaStream_t s = own_stream ? own_stream : s_caller;  // copies ordered after the allocation
  for (int l = 0; l <= L; ++l) {
    const Level& LV = lev[l];
    for (auto pr : {std::make_pair(&LV.E, &LV.E2), std::make_pair(&LV.F, &LV.F2), std::make_pair(&LV.G, &LV.G2)}) {
      pr.second->alloc(pr.first->n);
      copy_d2df(pr.first->p, pr.second->p, pr.first->n, s);
    }
  }
  RW_CUDA(cudaStreamSynchronize(s));
  has_df_inv = true;
}

void Hbs::make_fp32_fwd(cudaStream_t s_caller) const {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (has_fp32_fwd) return;
  AllocStreamScope scope(own_stream);
  cudaStream_t s = own_stream ? own_stream : s_caller;  // copies ordered after the allocation
  for (int l = 0; l <= L; ++l) {
    const Level& LV = lev[l];
    for (auto pr : {std::make_pair(&LV.U, &LV.Uf), std::make_pair(&LV.Vt, &LV.Vtf), std::make_pair(&LV.B, &LV.Bf),
                    std::make_pair(&LV.D, &LV.Df)}) {
      pr.second->alloc(pr.first->n);
      copy_d2f(pr.first->p, pr.second->p, pr.first->n, s);
    }
  }
  RW_CUDA(cudaStreamSynchronize(s));
  has_fp32_fwd = true;
}

template <class MT>
void Hbs::forward_impl(const double* xin, double* y, int nrhs, cudaStream_t s) const {
  // matrices in MT: the FP64 factors, or their double-FP32 copies
  auto pick = [](const DBuf<double>& d, const DBuf<float2>& f) -> const MT* {
    if constexpr (std::is_same<MT, double>::value) return d.p;
    else return f.p;
  };
  typedef GemvProb<double, MT> GP;
  const int ld = 2 * N;
  if (L == 0) {
    matvec<double, MT>({GP{pick(lev[0].D, lev[0].D2), xin, y, ld, ld, ld, ld, ld, 1.0, 0.0}}, nrhs, s);
    return;
  }
  std::vector<TBuf<double>> xh(L + 1), yh(L + 1);
  for (int l = 1; l <= L; ++l) {
    const int K = lev[l].koff.back();
    xh[l] = TBuf<double>(size_t(K) * nrhs, s);
    yh[l] = TBuf<double>(size_t(K) * nrhs, s);
  }
  {
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const int K = LV.koff.back();
    std::vector<GP> ps;
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      ps.push_back(GP{pick(LV.Vt, LV.Vt2) + LV.oVt[t], xin + 2 * nd.lo, xh[l].p + LV.koff[t], nd.k, n, nd.k, ld, K, 1.0, 0.0});
      ps.push_back(GP{pick(LV.D, LV.D2) + LV.oD[t], xin + 2 * nd.lo, y + 2 * nd.lo, n, n, n, ld, ld, 1.0, 0.0});
    }
    matvec<double, MT>(ps, nrhs, s);
  }
  for (int l = L - 1; l >= 1; --l) {
    const int h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    const int K = LV.koff.back(), KC = LC.koff.back();
    std::vector<GP> ps;
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      ps.push_back(GP{pick(LV.Vt, LV.Vt2) + LV.oVt[t], xh[l + 1].p + LC.koff[2 * t], xh[l].p + LV.koff[t], nd.k, nd.m, nd.k, KC, K, 1.0, 0.0});
    }
    matvec<double, MT>(ps, nrhs, s);
  }
  // sibling interactions at every parent, then interpolation down
  for (int l = 0; l <= L - 1; ++l) {
    const int h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    const int KC = LC.koff.back();
    if (l >= 1) {
      const int K = LV.koff.back();
      std::vector<GP> ps;
      for (int t = 0; t < nn; ++t) {
        const HbsNode& nd = node[h0 + t];
        ps.push_back(GP{pick(LV.U, LV.U2) + LV.oU[t], yh[l].p + LV.koff[t], yh[l + 1].p + LC.koff[2 * t], nd.m, nd.k, nd.m, K, KC, 1.0, 0.0});
      }
      matvec<double, MT>(ps, nrhs, s);
    }
    std::vector<GP> ps;
    for (int t = 0; t < nn; ++t) {
      const HbsNode& a = node[2 * (h0 + t)];
      const HbsNode& b = node[2 * (h0 + t) + 1];
      const int ia = LC.koff[2 * t], ib = LC.koff[2 * t + 1];
      const double beta = (l >= 1) ? 1.0 : 0.0;
      ps.push_back(GP{pick(LV.B, LV.B2) + LV.oB12[t], xh[l + 1].p + ib, yh[l + 1].p + ia, a.k, b.k, a.k, KC, KC, 1.0, beta});
      ps.push_back(GP{pick(LV.B, LV.B2) + LV.oB21[t], xh[l + 1].p + ia, yh[l + 1].p + ib, b.k, a.k, b.k, KC, KC, 1.0, beta});
    }
    matvec<double, MT>(ps, nrhs, s);
  }
  {
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const int K = LV.koff.back();
    std::vector<GP> ps;
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      ps.push_back(GP{pick(LV.U, LV.U2) + LV.oU[t], yh[l].p + LV.koff[t], y + 2 * nd.lo, n, nd.k, n, K, ld, 1.0, 1.0});
    }
    matvec<double, MT>(ps, nrhs, s);
  }
}

}  // namespace rw
