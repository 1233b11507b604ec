// GEMM programs of one refinement (many right-hand sides): the extended
// system's operator A~ + L R (Eq. ELS_approximate), Algorithm 1's solve
// (Eq. wood) in FP64, and the low-precision preconditioner of Sec. 4.2.  The
// wall's tree, the refined arc's tree and the Woodbury products share phases,
// so a whole operator apply or solve is one persistent launch per 64
// right-hand sides.
#include "refine.cuh"

namespace rw {

namespace {

// R y with R = [[0, R_kc, R_kp], [R_pk, 0, 0]] on ext vectors (y_o at base
// yob, y_p at base ypb, ld 2No / 2Np), into r (base rb, offset ro, ld rld):
// phases p (gather of the cut rows, R_pk y_o), p + 1 (R_kc y_c), p + 2
// (R_kp y_p).  Returns the next free phase.
template <class GP, class MT>
int emit_r_times(GP& P, int p, const MT* Rkc, const MT* Rkp, const MT* Rpk, int kk, int kpk, int k, int No, int Nc,
                 int Np, const int* dc, int yob, int ypb, int rb, long long ro, int rld) {
  const int W = P.ws_base();
  const long long yc = P.ws_alloc(std::max(2LL * Nc, 1LL));
  if (Nc) P.copy(p, 2 * Nc, yob, 0, 2 * No, dc, W, yc, -1, nullptr);
  if (kpk) P.gemm(p, Rpk, kpk, 2 * No, kpk, yob, 0, 2 * No, rb, ro + kk, rld, 1.0, 0.0);
  if (kk && Nc) P.gemm(p + 1, Rkc, kk, 2 * Nc, kk, W, yc, -1, rb, ro, rld, 1.0, 0.0);
  if (kk && Np) P.gemm(p + 2, Rkp, kk, 2 * Np, kk, ypb, 0, 2 * Np, rb, ro, rld, 1.0, Nc ? 1.0 : 0.0);
  (void)k;
  return p + 3;
}

}  // namespace

const GProgram<double>& Refinement::els_prog(bool df, cudaStream_t s) const {
  GProgram<double>& P = df ? g_elsdf : g_els64;
  if (P.finalized()) return P;
  if (df) {
    make_mixed();
    wall->op().make_df(s);
  }
  const int at = df ? MA_DF : MA_F64;
  const int pw = wall->op().emit_forward_g(P, 0, 0, 0, 2 * No, 3, 0, 2 * No, at);
  const int pp = hpp.emit_forward_g(P, 0, 1, 0, 2 * Np, 4, 0, 2 * Np, at);
  if (k > 0) {
    const long long r = P.ws_alloc(k);
    int q;
    if (df) q = emit_r_times(P, 0, Rkc2.p, Rkp2.p, Rpk2.p, kk, kpk, k, No, Nc, Np, dc.p, 0, 1, P.ws_base(), r, -1);
    else q = emit_r_times(P, 0, Rkc.p, Rkp.p, Rpk.p, kk, kpk, k, No, Nc, Np, dc.p, 0, 1, P.ws_base(), r, -1);
    q = std::max(q, std::max(pw, pp));
    if (df) {
      if (kk) P.gemm(q, Lo2.p, 2 * No, kk, 2 * No, P.ws_base(), r, -1, 3, 0, 2 * No, 1.0, 1.0);
      if (kpk) P.gemm(q, Lp2.p, 2 * Np, kpk, 2 * Np, P.ws_base(), r + kk, -1, 4, 0, 2 * Np, 1.0, 1.0);
    } else {
      if (kk) P.gemm(q, Lo.p, 2 * No, kk, 2 * No, P.ws_base(), r, -1, 3, 0, 2 * No, 1.0, 1.0);
      if (kpk) P.gemm(q, Lp.p, 2 * Np, kpk, 2 * Np, P.ws_base(), r + kk, -1, 4, 0, 2 * Np, 1.0, 1.0);
    }
  }
  P.finalize(s, streams.main);
  return P;
}

const GProgram<float>& Refinement::els_prog32(cudaStream_t s) const {
  GProgram<float>& P = g_els32;
  if (P.finalized()) return P;
  make_mixed();
  wall->op().make_fp32_fwd(s);
  const int pw = wall->op().emit_forward_g(P, 0, 0, 0, 2 * No, 3, 0, 2 * No, MA_F32);
  const int pp = hpp.emit_forward_g(P, 0, 1, 0, 2 * Np, 4, 0, 2 * Np, MA_F32);
  if (k > 0) {
    const long long r = P.ws_alloc(k);
    int q = emit_r_times(P, 0, Rkc32.p, Rkp32.p, Rpk32.p, kk, kpk, k, No, Nc, Np, dc.p, 0, 1, P.ws_base(), r, -1);
    q = std::max(q, std::max(pw, pp));
    if (kk) P.gemm(q, Lo32.p, 2 * No, kk, 2 * No, P.ws_base(), r, -1, 3, 0, 2 * No, 1.0, 1.0);
    if (kpk) P.gemm(q, Lp32.p, 2 * Np, kpk, 2 * Np, P.ws_base(), r + kk, -1, 4, 0, 2 * Np, 1.0, 1.0);
  }
  P.finalize(s, streams.main);
  return P;
}

namespace {
// Algorithm 1's Woodbury correction after the sweeps (which end before phase
// p0): r = R y, z = W^{-1} r, y -= X z (Eq. wood); factors of one type MT.
template <class MT>
void emit_woodbury(GProgram<double>& P, int p0, const MT* Rkc, const MT* Rkp, const MT* Rpk, const MT* Winv,
                   const MT* Xo, const MT* Xp, int kk, int kpk, int k, int No, int Nc, int Np, const int* dc) {
  const int W = P.ws_base();
  const long long r = P.ws_alloc(k), z = P.ws_alloc(k);
  int p = emit_r_times(P, p0, Rkc, Rkp, Rpk, kk, kpk, k, No, Nc, Np, dc, 3, 4, W, r, -1);
  P.gemm(p, Winv, k, k, k, W, r, -1, W, z, -1, 1.0, 0.0);
  ++p;
  if (kk) P.gemm(p, Xo, 2 * No, kk, 2 * No, W, z, -1, 3, 0, 2 * No, -1.0, 1.0);
  if (kpk) P.gemm(p, Xp, 2 * Np, kpk, 2 * Np, W, z + kk, -1, 4, 0, 2 * Np, -1.0, 1.0);
}
}  // namespace

const GProgram<double>& Refinement::dir_prog(cudaStream_t s, bool df) const {
  GProgram<double>& P = df ? g_dirdf : g_dir64;
  if (P.finalized()) return P;
  if (df) {
    make_mixed();
    wall->hbs.make_df_inv(s);
    hpp.make_df_inv(s);
  }
  const int at = df ? MA_DF : MA_F64;
  const int pa = wall->hbs.emit_inverse_g(P, 0, 0, 0, 2 * No, 3, 0, 2 * No, at);
  const int pb = hpp.emit_inverse_g(P, 0, 1, 0, 2 * Np, 4, 0, 2 * Np, at);
  if (k > 0) {
    if (df)
      emit_woodbury(P, std::max(pa, pb), Rkc2.p, Rkp2.p, Rpk2.p, Winv2.p, Xo2.p, Xp2.p, kk, kpk, k, No, Nc, Np, dc.p);
    else
      emit_woodbury(P, std::max(pa, pb), Rkc.p, Rkp.p, Rpk.p, Winv.p, Xo.p, Xp.p, kk, kpk, k, No, Nc, Np, dc.p);
  }
  P.finalize(s, streams.main);
  return P;
}

const GProgram<float>& Refinement::pre_prog_a(bool bf16, cudaStream_t s) const {
  GProgram<float>& P = bf16 ? g_pre16 : g_pre32;
  if (P.finalized()) return P;
  make_mixed();
  const int at = bf16 ? MA_BF16 : MA_F32;
  const int pa = wall->hbs.emit_inverse_g(P, 0, 0, 0, 2 * No, 3, 0, 2 * No, at);
  const int pb = hpp.emit_inverse_g(P, 0, 1, 0, 2 * Np, 4, 0, 2 * Np, at);
  if (k > 0)
    emit_r_times(P, std::max(pa, pb), Rkc32.p, Rkp32.p, Rpk32.p, kk, kpk, k, No, Nc, Np, dc.p, 3, 4, 5, 0, k);
  P.finalize(s, streams.main);
  return P;
}

const GProgram<float>& Refinement::pre_prog_b(cudaStream_t s) const {
  GProgram<float>& P = g_preb;
  if (P.finalized()) return P;
  make_mixed();
  if (kk) P.gemm(0, Xo32.p, 2 * No, kk, 2 * No, 5, 0, k, 3, 0, 2 * No, -1.0, 1.0);
  if (kpk) P.gemm(0, Xp32.p, 2 * Np, kpk, 2 * Np, 5, kk, k, 4, 0, 2 * Np, -1.0, 1.0);
  P.finalize(s, streams.main);
  return P;
}

template <class T>
void run_prog(const GProgram<T>& P, const T* b0, const T* b1, T* b3, T* b4, T* b5, int nrhs, cudaStream_t s) {
  TBuf<T> ws(size_t(std::max<long long>(P.ws_per_rhs(), 1)) * nrhs, s);
  T* bases[kGBases] = {const_cast<T*>(b0), const_cast<T*>(b1), ws.p, b3, b4, b5};
  P.run(bases, nrhs, s);
}
template void run_prog<double>(const GProgram<double>&, const double*, const double*, double*, double*, double*, int,
                               cudaStream_t);
template void run_prog<float>(const GProgram<float>&, const float*, const float*, float*, float*, float*, int,
                              cudaStream_t);

}  // namespace rw
