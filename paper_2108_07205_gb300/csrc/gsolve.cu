// HBS forward apply and inverse sweep as GEMM programs (many right-hand
// sides), and the cached single-launch versions on a handle.
//
// Forward apply y = A x of the HBS representation (Sec. 3 preamble; GYM
// 2012): up the tree the skeleton values xh = V* x (leaves) and xh_parent =
// V* [xh_a; xh_b]; across each pair of siblings yh_a = B12 xh_b, yh_b = B21
// xh_a; down the tree yh_children += U yh_parent; at the leaves y = D x +
// U yh.  Phases (a product runs as soon as its inputs are final):
//   0            leaves: xh_L = V* x, y = D x
//   L - l        up (l >= 1): xh_l = V* xh_{l+1};  siblings of level l: yh_{l+1} = B xh_{l+1}
//   L + l        down (1 <= l < L): yh_{l+1} += U yh_l
//   2L           leaves: y += U yh_L
// Inverse sweep x = A^{-1} b (F* up, G at every level, E down), phases
//   0            leaves: uh_L = F* b, x = G b
//   L - l        up (l >= 1): uh_l = F* uh_{l+1}, qh_{l+1} = G uh_{l+1}
//   L            root: qh_1 = G_0 uh_1
//   L + l        down (1 <= l < L): qh_{l+1} += E qh_l
//   2L           leaves: x += E qh_L
#include "hbs.cuh"
#include <functional>
#include <mutex>

namespace rw {

namespace {

// Factor pointer of a level by arithmetic.
template <class D, class F, class H, class P2>
const void* pick_ptr(int atype, const D& d64, const F* d32, const H* d16, const P2* d2) {
  switch (atype) {
    case MA_F32: return d32 ? static_cast<const void*>(d32->p) : nullptr;
    case MA_BF16: return d16 ? static_cast<const void*>(d16->p) : nullptr;
    case MA_DF: return d2 ? static_cast<const void*>(d2->p) : nullptr;
    default: return static_cast<const void*>(d64.p);
  }
}

template <class GP>
void put(GP& P, int p, const void* base, int atype, size_t off, int m, int n, int lda, int xb, long long xo, int ldx,
         int yb, long long yo, int ldy, double alpha, double beta) {
  require(base != nullptr || m * n == 0, "GEMM program: factor copy of this precision missing");
  switch (atype) {
    case MA_F32:
      P.gemm(p, static_cast<const float*>(base) + off, m, n, lda, xb, xo, ldx, yb, yo, ldy, alpha, beta);
      break;
    case MA_BF16:
      P.gemm(p, static_cast<const __nv_bfloat16*>(base) + off, m, n, lda, xb, xo, ldx, yb, yo, ldy, alpha, beta);
      break;
    case MA_DF:
      P.gemm(p, static_cast<const float2*>(base) + off, m, n, lda, xb, xo, ldx, yb, yo, ldy, alpha, beta);
      break;
    default:
      P.gemm(p, static_cast<const double*>(base) + off, m, n, lda, xb, xo, ldx, yb, yo, ldy, alpha, beta);
  }
}

}  // namespace

template <class GP>
int Hbs::emit_forward_g(GP& P, int p0, int xb, long long xo, int ldx, int yb, long long yo, int ldy, int atype) const {
  const int W = P.ws_base();
  auto U = [&](const Level& LV) { return pick_ptr(atype, LV.U, &LV.Uf, (const DBuf<__nv_bfloat16>*)nullptr, &LV.U2); };
  auto Vt = [&](const Level& LV) { return pick_ptr(atype, LV.Vt, &LV.Vtf, (const DBuf<__nv_bfloat16>*)nullptr, &LV.Vt2); };
  auto Bm = [&](const Level& LV) { return pick_ptr(atype, LV.B, &LV.Bf, (const DBuf<__nv_bfloat16>*)nullptr, &LV.B2); };
  auto Dm = [&](const Level& LV) { return pick_ptr(atype, LV.D, &LV.Df, (const DBuf<__nv_bfloat16>*)nullptr, &LV.D2); };
  if (L == 0) {
    const int n = 2 * N;
    put(P, p0, Dm(lev[0]), atype, 0, n, n, n, xb, xo, ldx, yb, yo, ldy, 1.0, 0.0);
    return p0 + 1;
  }
  std::vector<long long> xh(L + 1), yh(L + 1);
  for (int l = 1; l <= L; ++l) {
    xh[l] = P.ws_alloc(lev[l].koff.back());
    yh[l] = P.ws_alloc(lev[l].koff.back());
  }
  {  // leaves
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      put(P, p0, Vt(LV), atype, LV.oVt[t], nd.k, n, nd.k, xb, xo + 2 * nd.lo, ldx, W, xh[l] + LV.koff[t], -1, 1.0, 0.0);
      put(P, p0, Dm(LV), atype, LV.oD[t], n, n, n, xb, xo + 2 * nd.lo, ldx, yb, yo + 2 * nd.lo, ldy, 1.0, 0.0);
    }
  }
  for (int l = L - 1; l >= 0; --l) {
    const int p = p0 + (L - l), h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      if (l >= 1)
        put(P, p, Vt(LV), atype, LV.oVt[t], nd.k, nd.m, nd.k, W, xh[l + 1] + LC.koff[2 * t], -1, W,
            xh[l] + LV.koff[t], -1, 1.0, 0.0);
      const HbsNode& a = node[2 * (h0 + t)];
      const HbsNode& b = node[2 * (h0 + t) + 1];
      const long long ia = LC.koff[2 * t], ib = LC.koff[2 * t + 1];
      put(P, p, Bm(LV), atype, LV.oB12[t], a.k, b.k, a.k, W, xh[l + 1] + ib, -1, W, yh[l + 1] + ia, -1, 1.0, 0.0);
      put(P, p, Bm(LV), atype, LV.oB21[t], b.k, a.k, b.k, W, xh[l + 1] + ia, -1, W, yh[l + 1] + ib, -1, 1.0, 0.0);
    }
  }
  for (int l = 1; l <= L - 1; ++l) {
    const int p = p0 + L + l, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      put(P, p, U(LV), atype, LV.oU[t], nd.m, nd.k, nd.m, W, yh[l] + LV.koff[t], -1, W, yh[l + 1] + LC.koff[2 * t], -1,
          1.0, 1.0);
    }
  }
  {
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      put(P, p0 + 2 * L, U(LV), atype, LV.oU[t], n, nd.k, n, W, yh[l] + LV.koff[t], -1, yb, yo + 2 * nd.lo, ldy, 1.0,
          1.0);
    }
  }
  return p0 + 2 * L + 1;
}

template <class GP>
int Hbs::emit_inverse_g(GP& P, int p0, int xb, long long xo, int ldx, int yb, long long yo, int ldy, int atype) const {
  const int W = P.ws_base();
  auto Fm = [&](const Level& LV) { return pick_ptr(atype, LV.F, &LV.F32, &LV.F16, &LV.F2); };
  auto Gm = [&](const Level& LV) { return pick_ptr(atype, LV.G, &LV.G32, &LV.G16, &LV.G2); };
  auto Em = [&](const Level& LV) { return pick_ptr(atype, LV.E, &LV.E32, &LV.E16, &LV.E2); };
  if (L == 0) {
    const int n = 2 * N;
    put(P, p0, Gm(lev[0]), atype, 0, n, n, n, xb, xo, ldx, yb, yo, ldy, 1.0, 0.0);
    return p0 + 1;
  }
  std::vector<long long> uh(L + 1), qh(L + 1);
  for (int l = 1; l <= L; ++l) {
    uh[l] = P.ws_alloc(lev[l].koff.back());
    qh[l] = P.ws_alloc(lev[l].koff.back());
  }
  {  // leaves: uh = F* b, x = G b
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      put(P, p0, Fm(LV), atype, LV.oF[t], nd.k, n, nd.k, xb, xo + 2 * nd.lo, ldx, W, uh[l] + LV.koff[t], -1, 1.0, 0.0);
      put(P, p0, Gm(LV), atype, LV.oG[t], n, n, n, xb, xo + 2 * nd.lo, ldx, yb, yo + 2 * nd.lo, ldy, 1.0, 0.0);
    }
  }
  for (int l = L - 1; l >= 1; --l) {
    const int p = p0 + (L - l), h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const long long in = uh[l + 1] + LC.koff[2 * t];
      put(P, p, Fm(LV), atype, LV.oF[t], nd.k, nd.m, nd.k, W, in, -1, W, uh[l] + LV.koff[t], -1, 1.0, 0.0);
      put(P, p, Gm(LV), atype, LV.oG[t], nd.m, nd.m, nd.m, W, in, -1, W, qh[l + 1] + LC.koff[2 * t], -1, 1.0, 0.0);
    }
  }
  {
    const int K1 = lev[1].koff.back();
    put(P, p0 + L, Gm(lev[0]), atype, 0, K1, K1, K1, W, uh[1], -1, W, qh[1], -1, 1.0, 0.0);
  }
  for (int l = 1; l <= L - 1; ++l) {
    const int p = p0 + L + l, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    const Level& LC = lev[l + 1];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      put(P, p, Em(LV), atype, LV.oE[t], nd.m, nd.k, nd.m, W, qh[l] + LV.koff[t], -1, W, qh[l + 1] + LC.koff[2 * t],
          -1, 1.0, 1.0);
    }
  }
  {
    const int l = L, h0 = 1 << l, nn = 1 << l;
    const Level& LV = lev[l];
    for (int t = 0; t < nn; ++t) {
      const HbsNode& nd = node[h0 + t];
      const int n = 2 * (nd.hi - nd.lo);
      put(P, p0 + 2 * L, Em(LV), atype, LV.oE[t], n, nd.k, n, W, qh[l] + LV.koff[t], -1, yb, yo + 2 * nd.lo, ldy, 1.0,
          1.0);
    }
  }
  return p0 + 2 * L + 1;
}

template int Hbs::emit_forward_g<GProgram<double>>(GProgram<double>&, int, int, long long, int, int, long long, int,
                                                   int) const;
template int Hbs::emit_inverse_g<GProgram<double>>(GProgram<double>&, int, int, long long, int, int, long long, int,
                                                   int) const;
template int Hbs::emit_forward_g<GProgram<float>>(GProgram<float>&, int, int, long long, int, int, long long, int,
                                                  int) const;
template int Hbs::emit_inverse_g<GProgram<float>>(GProgram<float>&, int, int, long long, int, int, long long, int,
                                                  int) const;

namespace {
std::mutex g_prog_mu;  // cached programs of a wall may be asked for by several serving workers
}

// Cached one-launch programs on the handle: bases 0 = input, 1 = output,
// 2 = workspace.
template <class T>
static void run_cached(GProgram<T>& prog, const std::function<void(GProgram<T>&)>& emit, const T* in, T* out,
                       int nrhs, cudaStream_t alloc, cudaStream_t s) {
  {
    std::lock_guard<std::mutex> lock(g_prog_mu);
    if (!prog.finalized()) {
      emit(prog);
      prog.finalize(s, alloc);
    }
  }
  TBuf<T> ws(size_t(std::max<long long>(prog.ws_per_rhs(), 1)) * nrhs, s);
  T* bases[kGBases] = {const_cast<T*>(in), out, ws.p, nullptr, nullptr, nullptr};
  prog.run(bases, nrhs, s);
}

void Hbs::forward_gemm(const double* x, double* y, int nrhs, bool df, cudaStream_t s) const {
  if (df) make_df(s);
  GProgram<double>& P = df ? gfwddf : gfwd64;
  run_cached<double>(P, [&](GProgram<double>& G) {
    emit_forward_g(G, 0, 0, 0, 2 * N, 1, 0, 2 * N, df ? MA_DF : MA_F64);
  }, x, y, nrhs, own_stream, s);
}

void Hbs::inverse_gemm(const double* b, double* x, int nrhs, cudaStream_t s) const {
  run_cached<double>(ginv64, [&](GProgram<double>& G) { emit_inverse_g(G, 0, 0, 0, 2 * N, 1, 0, 2 * N, MA_F64); },
                     b, x, nrhs, own_stream, s);
}

void Hbs::inverse_gemm_df(const double* b, double* x, int nrhs, cudaStream_t s) const {
  make_df_inv(s);
  run_cached<double>(ginvdf, [&](GProgram<double>& G) { emit_inverse_g(G, 0, 0, 0, 2 * N, 1, 0, 2 * N, MA_DF); },
                     b, x, nrhs, own_stream, s);
}

void Hbs::inverse_gemm_f32(const float* b, float* x, int nrhs, bool bf16, cudaStream_t s) const {
  require(bf16 ? has_bf16 : has_fp32, "HBS: low-precision copies not built");
  GProgram<float>& P = bf16 ? ginv16 : ginv32;
  run_cached<float>(P, [&](GProgram<float>& G) {
    emit_inverse_g(G, 0, 0, 0, 2 * N, 1, 0, 2 * N, bf16 ? MA_BF16 : MA_F32);
  }, b, x, nrhs, own_stream, s);
}

}  // namespace rw
