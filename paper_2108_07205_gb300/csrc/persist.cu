// Checkpoint and restore of a built wall (rw_hbs_save / rw_hbs_load): the
// curve, options, nodes, HBS tree (ranges, ranks, skeletons) and every
// forward and inverse factor, so that a restored handle gives the same results
// as the one saved without repeating the build.  The FP32 copies of the
// inverse factors are rebuilt on load.  Format: an 8-byte tag and version,
// then little-endian fields and length-prefixed arrays in a fixed order.
#include "handles.cuh"
#include <cstdio>
#include <cstring>
#include <memory>

namespace {

constexpr char kTag[8] = {'R', 'W', 'H', 'B', 'S', 'v', '0', '2'};  // v02: options gained hole_div_ratio

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
  template <class T> void dbuf(rw::DBuf<T>& b) {
    const std::vector<T> h = vec<T>();
    b.alloc(h.size());
    if (!h.empty()) RW_CUDA(cudaMemcpy(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  }
};

void save_wall(const rw::Wall& w, Writer& o, cudaStream_t s) {
  o.raw(kTag, sizeof(kTag));
  o.val(w.curve.kind);
  for (double p : w.curve.p) o.val(p);
  o.val(w.n_panels);
  o.val(w.opts);
  o.val(w.nodes.n);
  o.dbuf(w.nodes.buf, s);
  const rw::Hbs& H = w.hbs;
  o.val(H.N);
  o.val(H.L);
  o.val(H.max_rank);
  o.val(H.inv_elems);
  o.val(H.fwd_elems);
  o.val((long long)H.bytes);
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
  o.raw(kTag, sizeof(kTag));  // trailer: a truncated file fails to load
}

void load_wall(rw::Wall& w, Reader& in, cudaStream_t s) {
  char tag[8];
  in.raw(tag, sizeof(tag));
  rw::require(std::memcmp(tag, kTag, sizeof(tag)) == 0, "rw_hbs_load: not a wall file of this version");
  w.curve.kind = in.val<int>();
  for (double& p : w.curve.p) p = in.val<double>();
  w.n_panels = in.val<int>();
  w.opts = in.val<rw::Opts>();
  const int n = in.val<int>();
  rw::require(n >= 16 && n == 16 * w.n_panels, "rw_hbs_load: corrupt node count");
  w.nodes.n = n;
  in.dbuf(w.nodes.buf);
  rw::require(w.nodes.buf.n == size_t(6) * n, "rw_hbs_load: corrupt node array");
  {
    const auto all = w.nodes.buf.download(s);
    w.nodes.hx.assign(all.begin(), all.begin() + n);
    w.nodes.hy.assign(all.begin() + n, all.begin() + 2 * size_t(n));
  }
  rw::Hbs& H = w.hbs;
  H.N = in.val<int>();
  H.L = in.val<int>();
  H.max_rank = in.val<int>();
  H.inv_elems = in.val<long long>();
  H.fwd_elems = in.val<long long>();
  H.bytes = size_t(in.val<long long>());
  rw::require(H.N == n && H.L >= 0 && H.L <= 24, "rw_hbs_load: corrupt tree header");
  const long long nn = in.val<long long>();
  rw::require(nn == (2LL << H.L), "rw_hbs_load: corrupt tree size");
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
  rw::require(nl == H.L + 1, "rw_hbs_load: corrupt level count");
  H.lev.clear();
  H.lev.resize(size_t(nl));
  for (auto& LV : H.lev) {
    for (auto* b : {&LV.U, &LV.Vt, &LV.E, &LV.F, &LV.G, &LV.B, &LV.D}) in.dbuf(*b);
    for (auto* v : {&LV.oU, &LV.oVt, &LV.oE, &LV.oF, &LV.oG, &LV.oB12, &LV.oB21, &LV.oD}) *v = in.vec<size_t>();
    LV.koff = in.vec<int>();
  }
  in.raw(tag, sizeof(tag));
  rw::require(std::memcmp(tag, kTag, sizeof(tag)) == 0, "rw_hbs_load: corrupt trailer");
  H.make_fp32(s);
  H.make_bf16(s);
  RW_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

extern "C" {

int rw_hbs_save(rw_hbs_t h, const char* path) {
  if (!h || !path) return rw::abi_fail(RW_ERR_INVALID, "rw_hbs_save: null argument");
  try {
    File f(path, "wb");
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
