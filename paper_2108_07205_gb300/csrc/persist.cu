// Checkpoint and restore of a built wall (rw_hbs_save / rw_hbs_load): the
// curve, options, nodes, HBS tree (ranges, ranks, skeletons) and every
// forward and inverse factor, so that a restored handle gives the same results
// as the one saved without repeating the build.  The FP32 copies of the
// inverse factors are rebuilt on load.  Format: an 8-byte tag and version,
// then little-endian fields and length-prefixed arrays in a fixed order.
#include "handles.cuh"
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>

namespace {

// v04: options gained op_tol and mixed_factor, and the wall may carry a second
// (forward-only) HBS at op_tol
constexpr char kTag[8] = {'R', 'W', 'H', 'B', 'S', 'v', '0', '4'};

struct File {
  FILE* f = nullptr;
  File(const char* path, const char* mode) : f(std::fopen(path, mode)) {}
  ~File() { if (f) std::fclose(f); }
};

struct Writer {
  FILE* f;
  void raw(const void* p, size_t n) {
    if (n && std::fwrite(p, 1, n, f) != n) throw rw::Error(RW_ERR_INVALID, "rw_hbs_save: write failed");
  }
  template <class T> void val(const T& v) { raw(&v, sizeof(T)); }
  template <class T> void vec(const std::vector<T>& v) {
    val<long long>((long long)v.size());
    raw(v.data(), v.size() * sizeof(T));
  }
  template <class T> void dbuf(const rw::DBuf<T>& b, cudaStream_t s) { vec(b.download(s)); }
};

struct Reader {
  FILE* f;
  void raw(void* p, size_t n) {
    if (n && std::fread(p, 1, n, f) != n) throw rw::Error(RW_ERR_INVALID, "rw_hbs_load: truncated file");
  }
  template <class T> T val() {
    T v;
    raw(&v, sizeof(T));
    return v;
  }
  template <class T> std::vector<T> vec() {
    const long long n = val<long long>();
    rw::require(n >= 0 && n <= (1LL << 36) / (long long)sizeof(T), "rw_hbs_load: corrupt array length");
    std::vector<T> v(static_cast<size_t>(n));
    raw(v.data(), v.size() * sizeof(T));
    return v;
  }
};

void save_hbs(const rw::Hbs& H, Writer& o, cudaStream_t s) {
  o.val(H.N);
  o.val(H.L);
  o.val((long long)H.node.size());
  for (const rw::HbsNode& nd : H.node) {
    o.val(nd.lo);
    o.val(nd.hi);
    o.val(nd.k);
    o.val(nd.m);
    o.vec(nd.skr);
    o.vec(nd.skc);
  }
  o.val((long long)H.lev.size());
  for (const auto& LV : H.lev) {
    for (const auto* b : {&LV.U, &LV.Vt, &LV.E, &LV.F, &LV.G, &LV.B, &LV.D}) o.dbuf(*b, s);
    for (const auto* v : {&LV.oU, &LV.oVt, &LV.oE, &LV.oF, &LV.oG, &LV.oB12, &LV.oB21, &LV.oD}) o.vec(*v);
    o.vec(LV.koff);
  }
}

void save_wall(const rw::Wall& w, Writer& o, cudaStream_t s) {
  o.raw(kTag, sizeof(kTag));
  o.val(w.curve.kind);
  for (double p : w.curve.p) o.val(p);
  o.val(w.n_panels);
  o.val(w.opts);
  o.val(w.nodes.n);
  o.dbuf(w.nodes.buf, s);
  save_hbs(w.hbs, o, s);
  o.val<int>(w.hbs_op.N ? 1 : 0);
  if (w.hbs_op.N) save_hbs(w.hbs_op, o, s);
  o.raw(kTag, sizeof(kTag));  // trailer: a truncated file fails to load
}

// The options as rw_hbs_build accepts them (a damaged file must not smuggle
// in sizes the kernels were never meant to see).
void check_opts(const rw::Opts& o) {
  auto fin = [](double v) { return std::isfinite(v); };
  rw::require(o.leaf_points >= 8 && o.leaf_points <= 512 && fin(o.id_tol) && o.id_tol > 0 && o.id_tol < 1 &&
                  o.n_proxy >= 8 && o.n_proxy <= 1024 && fin(o.proxy_ratio) && o.proxy_ratio > 1.0 &&
                  o.n_proxy_refine >= 8 && o.n_proxy_refine <= 1024 && fin(o.div_ratio) && fin(o.bas_ratio) &&
                  o.div_ratio > o.bas_ratio && o.bas_ratio > 1.0 && fin(o.hole_div_ratio) &&
                  o.hole_div_ratio > o.bas_ratio && o.sketch_cols >= 64 && o.sketch_width >= 16 &&
                  o.sketch_width <= 4096 && fin(o.gmres_tol) && o.gmres_tol > 0 && o.gmres_maxit >= 1 &&
                  o.gmres_maxit <= 10000 && o.gmres_restarts >= 1 && o.gmres_restarts <= 10000 &&
                  fin(o.op_tol) && o.op_tol >= 0 && o.op_tol < 1 && (o.mixed_factor >= 0 && o.mixed_factor <= 2),
              "rw_hbs_load: corrupt options");
}

// Host image of one HBS level as read from a file, checked before any of it
// reaches the device.
struct HostLevel {
  std::vector<double> buf[7];          // U, Vt, E, F, G, B, D
  std::vector<size_t> off[8];          // oU, oVt, oE, oF, oG, oB12, oB21, oD
  std::vector<int> koff;
};

void need(bool ok, const char* what) {
  if (!ok) throw rw::Error(RW_ERR_INVALID, std::string("rw_hbs_load: corrupt ") + what);
}

// Every block a sweep or an apply addresses must lie inside its buffer:
// off + rows * cols <= size, in 64-bit arithmetic.
void need_block(const std::vector<size_t>& off, size_t t, long long rows, long long cols, size_t size,
                const char* what) {
  need(t < off.size(), what);
  need(rows >= 0 && cols >= 0, what);
  const unsigned long long extent = (unsigned long long)rows * (unsigned long long)cols;
  need(off[t] <= size && extent <= size - off[t], what);
}

// Tree and factor checks: node ranges tile their parents, ranks and
// candidate counts are consistent, skeleton indices are DOFs of the wall, the
// offset tables have one entry per node and every block fits its buffer.
void check_hbs(const rw::Hbs& H, const std::vector<HostLevel>& hl, bool fwd_only) {
  const int N = H.N, L = H.L;
  const size_t nn_all = H.node.size();
  need(nn_all == (size_t(2) << L), "tree size");
  need(H.node[1].lo == 0 && H.node[1].hi == N, "root range");
  for (size_t h = 1; h < nn_all; ++h) {
    const rw::HbsNode& nd = H.node[h];
    need(nd.lo >= 0 && nd.lo < nd.hi && nd.hi <= N, "node range");
    if (2 * h + 1 < nn_all) {
      const rw::HbsNode& a = H.node[2 * h];
      const rw::HbsNode& b = H.node[2 * h + 1];
      need(a.lo == nd.lo && a.hi == b.lo && b.hi == nd.hi, "node ranges (children do not tile the parent)");
    }
  }
  for (int l = 0; l <= L; ++l) {
    const HostLevel& LV = hl[l];
    const int nn = 1 << l, h0 = 1 << l;
    const size_t sU = LV.buf[0].size(), sVt = LV.buf[1].size(), sE = LV.buf[2].size(), sF = LV.buf[3].size(),
                 sG = LV.buf[4].size(), sB = LV.buf[5].size(), sD = LV.buf[6].size();
    if (l >= 1) {
      need(LV.koff.size() == size_t(nn) + 1 && LV.koff[0] == 0, "rank offsets");
      need(LV.off[0].size() == size_t(nn) && LV.off[1].size() == size_t(nn), "U/V offsets");
      for (int t = 0; t < nn; ++t) {
        const rw::HbsNode& nd = H.node[h0 + t];
        const int m = (l == L) ? 2 * (nd.hi - nd.lo) : H.node[2 * (h0 + t)].k + H.node[2 * (h0 + t) + 1].k;
        need(nd.m == m && nd.k >= 0 && nd.k <= nd.m, "rank or candidate count");
        need((long long)LV.koff[t + 1] - LV.koff[t] == nd.k, "rank offsets");
        need(nd.skr.size() == size_t(nd.k) && nd.skc.size() == size_t(nd.k), "skeleton size");
        for (int d : nd.skr) need(d >= 2 * nd.lo && d < 2 * nd.hi, "skeleton index");
        for (int d : nd.skc) need(d >= 2 * nd.lo && d < 2 * nd.hi, "skeleton index");
        need_block(LV.off[0], t, nd.m, nd.k, sU, "U offset");
        need_block(LV.off[1], t, nd.k, nd.m, sVt, "V* offset");
        if (!fwd_only) {
          need_block(LV.off[2], t, nd.m, nd.k, sE, "E offset");
          need_block(LV.off[3], t, nd.k, nd.m, sF, "F* offset");
          need_block(LV.off[4], t, nd.m, nd.m, sG, "G offset");
        }
      }
    } else if (!fwd_only) {
      const int m0 = (L == 0) ? 2 * N : H.node[2].k + H.node[3].k;
      need_block(LV.off[4], 0, m0, m0, sG, "root G offset");
    }
    if (l < L) {
      for (int t = 0; t < nn; ++t) {
        const rw::HbsNode& a = H.node[2 * (h0 + t)];
        const rw::HbsNode& b = H.node[2 * (h0 + t) + 1];
        need_block(LV.off[5], t, a.k, b.k, sB, "B12 offset");
        need_block(LV.off[6], t, b.k, a.k, sB, "B21 offset");
      }
    } else {
      for (int t = 0; t < nn; ++t) {
        const rw::HbsNode& nd = H.node[h0 + t];
        const long long n = 2LL * (nd.hi - nd.lo);
        need_block(LV.off[7], t, n, n, sD, "leaf D offset");
      }
    }
  }
}

// Reads one HBS into H's tree fields and a host image of its factors, and
// checks them; nothing reaches the device here.
std::vector<HostLevel> parse_hbs(rw::Hbs& H, Reader& in, int n_points, bool fwd_only) {
  H.N = in.val<int>();
  H.L = in.val<int>();
  need(H.N == n_points && H.L >= 0 && H.L <= 20 && (H.N >> H.L) >= 1, "tree header");
  const long long nn = in.val<long long>();
  need(nn == (2LL << H.L), "tree size");
  H.node.assign(size_t(nn), rw::HbsNode());
  for (rw::HbsNode& nd : H.node) {
    nd.lo = in.val<int>();
    nd.hi = in.val<int>();
    nd.k = in.val<int>();
    nd.m = in.val<int>();
    nd.skr = in.vec<int>();
    nd.skc = in.vec<int>();
  }
  const long long nl = in.val<long long>();
  need(nl == H.L + 1, "level count");
  std::vector<HostLevel> hl(static_cast<size_t>(nl));
  for (auto& LV : hl) {
    for (auto& b : LV.buf) b = in.vec<double>();
    for (auto& v : LV.off) v = in.vec<size_t>();
    LV.koff = in.vec<int>();
  }
  check_hbs(H, hl, fwd_only);
  return hl;
}

// Uploads a checked host image and recomputes the statistics from it.
void upload_hbs(rw::Hbs& H, const std::vector<HostLevel>& hl) {
  H.lev.clear();
  H.lev.resize(hl.size());
  H.inv_elems = H.fwd_elems = 0;
  H.bytes = 0;
  H.max_rank = 0;
  for (size_t h = 2; h < H.node.size(); ++h) H.max_rank = std::max(H.max_rank, H.node[h].k);
  for (int l = 0; l <= H.L; ++l) {
    auto& LV = H.lev[l];
    rw::DBuf<double>* bufs[7] = {&LV.U, &LV.Vt, &LV.E, &LV.F, &LV.G, &LV.B, &LV.D};
    std::vector<size_t>* offs[8] = {&LV.oU, &LV.oVt, &LV.oE, &LV.oF, &LV.oG, &LV.oB12, &LV.oB21, &LV.oD};
    for (int q = 0; q < 7; ++q) {
      const auto& hb = hl[l].buf[q];
      bufs[q]->alloc(hb.size());
      if (!hb.empty()) RW_CUDA(cudaMemcpy(bufs[q]->p, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    for (int q = 0; q < 8; ++q) *offs[q] = hl[l].off[q];
    LV.koff = hl[l].koff;
    H.inv_elems += (long long)LV.G.n + (l > 0 ? (long long)LV.E.n + (long long)LV.F.n : 0);
    H.fwd_elems += (long long)LV.U.n * (l > 0) + (long long)LV.Vt.n * (l > 0) + (long long)LV.B.n * (l < H.L) +
                   (long long)LV.D.n;
    H.bytes += LV.U.bytes() + LV.Vt.bytes() + LV.E.bytes() + LV.F.bytes() + LV.G.bytes() + LV.B.bytes() +
               LV.D.bytes();
  }
}

// The whole file is read and checked before anything is uploaded, so a
// damaged file is refused with RW_ERR_INVALID and touches no device memory.
void load_wall(rw::Wall& w, Reader& in, cudaStream_t s) {
  char tag[8];
  in.raw(tag, sizeof(tag));
  rw::require(std::memcmp(tag, kTag, sizeof(tag)) == 0, "rw_hbs_load: not a wall file of this version");
  w.curve.kind = in.val<int>();
  need(w.curve.kind == RW_CURVE_STAR || w.curve.kind == RW_CURVE_CHANNEL || w.curve.kind == RW_CURVE_NODES,
       "curve kind");
  for (double& p : w.curve.p) {
    p = in.val<double>();
    need(std::isfinite(p), "curve parameters");
  }
  w.n_panels = in.val<int>();
  need(w.n_panels >= 1 && w.n_panels <= (1 << 20), "panel count");
  w.opts = in.val<rw::Opts>();
  check_opts(w.opts);
  const int n = in.val<int>();
  rw::require(n >= 16 && n == 16 * w.n_panels, "rw_hbs_load: corrupt node count");
  const std::vector<double> hn = in.vec<double>();
  need(hn.size() == size_t(6) * n, "node array");
  for (double v : hn) need(std::isfinite(v), "node array");
  const std::vector<HostLevel> h_main = parse_hbs(w.hbs, in, n, false);
  const int has_op = in.val<int>();
  need(has_op == (w.opts.factor_tol() < w.opts.id_tol ? 1 : 0), "operator flag");
  std::vector<HostLevel> h_op;
  if (has_op) h_op = parse_hbs(w.hbs_op, in, n, true);
  in.raw(tag, sizeof(tag));
  rw::require(std::memcmp(tag, kTag, sizeof(tag)) == 0, "rw_hbs_load: corrupt trailer");
  // upload
  w.nodes.n = n;
  w.nodes.buf.alloc(hn.size());
  RW_CUDA(cudaMemcpy(w.nodes.buf.p, hn.data(), hn.size() * sizeof(double), cudaMemcpyHostToDevice));
  w.nodes.hx.assign(hn.begin(), hn.begin() + n);
  w.nodes.hy.assign(hn.begin() + n, hn.begin() + 2 * size_t(n));
  upload_hbs(w.hbs, h_main);
  if (has_op) upload_hbs(w.hbs_op, h_op);
  w.hbs.make_fp32(s);
  w.hbs.make_bf16(s);
  RW_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

extern "C" {

int rw_hbs_save(rw_hbs_t h, const char* path) {
  if (!h || !path) return rw::abi_fail(RW_ERR_INVALID, "rw_hbs_save: null argument");
  try {
    File f(path, "wb");
    if (h->wall.nodes.kind == rw::kNodesExterior)
      throw rw::Error(RW_ERR_INVALID, "rw_hbs_save: exterior walls are not saved (rebuild them)");
    if (!f.f) throw rw::Error(RW_ERR_INVALID, std::string("rw_hbs_save: cannot open ") + path);
    Writer o{f.f};
    save_wall(h->wall, o, nullptr);
    if (std::fflush(f.f) != 0) throw rw::Error(RW_ERR_INVALID, "rw_hbs_save: write failed");
    rw::abi_clear_error();
    return RW_OK;
  } catch (const rw::Error& e) {
    return rw::abi_fail(e.code, e.what());
  } catch (const std::exception& e) {
    return rw::abi_fail(RW_ERR_INVALID, e.what());
  }
}

int rw_hbs_load(const char* path, void* stream, rw_hbs_t* out) {
  if (!path || !out) return rw::abi_fail(RW_ERR_INVALID, "rw_hbs_load: null argument");
  *out = nullptr;
  try {
    File f(path, "rb");
    if (!f.f) throw rw::Error(RW_ERR_INVALID, std::string("rw_hbs_load: cannot open ") + path);
    std::unique_ptr<rw_hbs_s> h(new rw_hbs_s);
    Reader in{f.f};
    load_wall(h->wall, in, static_cast<cudaStream_t>(stream));
    *out = h.release();
    rw::abi_clear_error();
    return RW_OK;
  } catch (const rw::Error& e) {
    return rw::abi_fail(e.code, e.what());
  } catch (const std::exception& e) {
    return rw::abi_fail(RW_ERR_INVALID, e.what());
  }
}

}  // extern "C"
