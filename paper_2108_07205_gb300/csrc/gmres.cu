// Mixed-precision path (Sec. 4.2): flexible GMRES in FP64 on the extended
// system (A~ + L R) tau_ext = g_ext (Eq. ELS_approximate), with A~ applied by
// the HBS forward representations of A_oo and A_pp and L R by its factors, all
// at the operator tolerance (op_tol).  The preconditioner is the Woodbury
// inverse of Sec. 4.2 whose A~^{-1} applications are HBS inverse sweeps in
// FP32 (or with the matrices in BF16, FP32 accumulation); W^{-1} stays FP64.
// In the mixed mode the operator's products run in double-FP32 (FP64-level
// accuracy on the FP32 units) and the preconditioner's Woodbury correction in
// FP32; otherwise they are FP64.
// Right preconditioning keeps the monitored residual equal to the true one.
// Every right-hand side runs its own Krylov space; the columns advance in
// lockstep and stop together once all have converged.
// Also the plain FP64 path to a certified residual: Algorithm 1 followed by
// FP64 iterative refinement against the same operator (solve_ir).
#include "refine.cuh"
#include <algorithm>
#include <cmath>

namespace rw {

namespace {

// out[c] = sum_i A[i, c] * B[i, c] (+ the same over a second row block), one
// CTA per column, fixed reduction order.
__global__ void k_coldot2(const double* A1, const double* B1, int n1, int ld1, const double* A2, const double* B2,
                          int n2, int ld2, int ncol_b, double* out) {
  // blockIdx.x = column c of A, blockIdx.y = basis vector index j (B offset j * ncol_b * ld)
  const int c = blockIdx.x, j = blockIdx.y;
  const double* a1 = A1 + size_t(c) * ld1;
  const double* b1 = B1 + (size_t(j) * ncol_b + c) * ld1;
  const double* a2 = A2 + size_t(c) * ld2;
  const double* b2 = B2 + (size_t(j) * ncol_b + c) * ld2;
  double s = 0.0;
  for (int i = threadIdx.x; i < n1; i += blockDim.x) s += a1[i] * b1[i];
  for (int i = threadIdx.x; i < n2; i += blockDim.x) s += a2[i] * b2[i];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[size_t(j) * gridDim.x + c] = red[0];
}

// Y[:, c] += sum_j coef[j * ncol + c] * B_j[:, c]  (nb basis vectors)
__global__ void k_colcomb(double* Y, const double* B, int n, int ld, int ncol, int nb, const double* coef) {
  const int c = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = Y[i + size_t(c) * ld];
    for (int j = 0; j < nb; ++j) acc += coef[size_t(j) * ncol + c] * B[i + (size_t(j) * ncol + c) * ld];
    Y[i + size_t(c) * ld] = acc;
  }
}

__global__ void k_colscale(const double* X, double* Y, int n, int ld, const double* sc) {
  const int c = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    Y[i + size_t(c) * ld] = X[i + size_t(c) * ld] * sc[c];
}

__global__ void k_d2f_v(const double* in, float* out, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) out[i] = float(in[i]);
}
__global__ void k_f2d_v(const float* in, double* out, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) out[i] = double(in[i]);
}

int g1(long long n) { return int(std::max<long long>(1, std::min<long long>((n + 255) / 256, 2048))); }

// Per-column squared norms (or dot products) of ext-space blocks, on the host.
std::vector<double> col_dots(const double* ao, const double* ap, const double* bo, const double* bp, int no, int np,
                             int nrhs, int nb, double* dots, cudaStream_t s) {
  k_coldot2<<<dim3(nrhs, nb), 256, 0, s>>>(ao, bo, no, no, ap, bp, np, np, nrhs, dots);
  RW_CHECK_LAUNCH();
  std::vector<double> h(size_t(nb) * nrhs);
  RW_CUDA(cudaMemcpyAsync(h.data(), dots, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  RW_CUDA(cudaStreamSynchronize(s));
  return h;
}

}  // namespace

void Refinement::make_mixed() const {
  if (has_mixed) return;
  cudaStream_t s = streams.main;
  AllocStreamScope scope(s);
  for (auto pr : {std::make_pair(&Lo, &Lo2), std::make_pair(&Lp, &Lp2), std::make_pair(&Rkc, &Rkc2),
                  std::make_pair(&Rkp, &Rkp2), std::make_pair(&Rpk, &Rpk2), std::make_pair(&Xo, &Xo2),
                  std::make_pair(&Xp, &Xp2), std::make_pair(&Winv, &Winv2)}) {
    if (pr.second->p && pr.second->n == pr.first->n) continue;  // made with W (see form_w)
    pr.second->alloc(pr.first->n);
    copy_d2df(pr.first->p, pr.second->p, pr.first->n, s);
  }
  for (auto pr : {std::make_pair(&Rkc, &Rkc32), std::make_pair(&Rkp, &Rkp32), std::make_pair(&Rpk, &Rpk32),
                  std::make_pair(&Xo, &Xo32), std::make_pair(&Xp, &Xp32), std::make_pair(&Lo, &Lo32),
                  std::make_pair(&Lp, &Lp32)}) {
    pr.second->alloc(pr.first->n);
    copy_d2f(pr.first->p, pr.second->p, pr.first->n, s);
  }
  hpp.make_df(s);
  hpp.make_fp32_fwd(s);
  RW_CUDA(cudaStreamSynchronize(s));
  has_mixed = true;
}

void Refinement::apply_els_df(const double* xo, const double* xp, double* yo, double* yp, int nrhs,
                              cudaStream_t s) const {
  make_mixed();
  if (nrhs > 8) {
    run_prog(els_prog(true, s), xo, xp, yo, yp, (double*)nullptr, nrhs, s);
    return;
  }
  wall->op().apply_forward_df(xo, yo, nrhs, s);
  hpp.apply_forward_df(xp, yp, nrhs, s);
  if (k == 0) return;
  typedef GemvProb<double, float2> GP;
  TBuf<double> xc(size_t(2) * Nc * nrhs, s), r(size_t(k) * nrhs, s);
  if (Nc) gather_scatter(xo, 2 * No, dc.p, xc.p, 2 * Nc, nullptr, 2 * Nc, nrhs, s);
  std::vector<GP> p1;
  if (kk && Nc) p1.push_back(GP{Rkc2.p, xc.p, r.p, kk, 2 * Nc, kk, 2 * Nc, k, 1.0, 0.0});
  if (kpk) p1.push_back(GP{Rpk2.p, xo, r.p + kk, kpk, 2 * No, kpk, 2 * No, k, 1.0, 0.0});
  matvec<double, float2>(p1, nrhs, s);
  if (kk && Np) matvec<double, float2>({GP{Rkp2.p, xp, r.p, kk, 2 * Np, kk, 2 * Np, k, 1.0, Nc ? 1.0 : 0.0}}, nrhs, s);
  std::vector<GP> p2;
  if (kk) p2.push_back(GP{Lo2.p, r.p, yo, 2 * No, kk, 2 * No, k, 2 * No, 1.0, 1.0});
  if (kpk) p2.push_back(GP{Lp2.p, r.p + kk, yp, 2 * Np, kpk, 2 * Np, k, 2 * Np, 1.0, 1.0});
  matvec<double, float2>(p2, nrhs, s);
}

void Refinement::solve_ir(const double* g, double* tau, int nrhs, cudaStream_t s, int* iters_out,
                          double* relres_out, bool df) const {
  const Opts& o = wall->opts;
  const int no = 2 * No, np = 2 * Np;
  TBuf<double> go(size_t(no) * nrhs, s), gp(size_t(np) * nrhs, s), xo(size_t(no) * nrhs, s), xp(size_t(np) * nrhs, s);
  TBuf<double> ro(size_t(no) * nrhs, s), rp(size_t(np) * nrhs, s), dso(size_t(no) * nrhs, s), dsp(size_t(np) * nrhs, s);
  TBuf<double> dots(size_t(nrhs), s);
  fill_zero(go.p, go.n, s);
  gather_scatter(g, 2 * Nn, n_from_o.p, go.p, no, n_to_o.p, nko, nrhs, s);
  gather_scatter(g, 2 * Nn, n_from_p.p, gp.p, np, n_to_p.p, nkp, nrhs, s);
  // Algorithm 1 in ext space: y = A~^{-1} v, then the Woodbury correction
  // (double-FP32: the GEMM programs at any nrhs)
  auto direct = [&](const double* vo, const double* vp, double* yo, double* yp) {
    if (df || nrhs > 8) {
      run_prog(dir_prog(s, df), vo, vp, yo, yp, (double*)nullptr, nrhs, s);
      return;
    }
    wall->hbs.apply_inverse_levels(vo, yo, nrhs, s);
    hpp.apply_inverse_levels(vp, yp, nrhs, s);
    woodbury_correct(yo, yp, nrhs, s);
  };
  direct(go.p, gp.p, xo.p, xp.p);
  std::vector<double> gn = col_dots(go.p, gp.p, go.p, gp.p, no, np, nrhs, 1, dots.p, s);
  int it = 0;
  double worst = 0.0;
  for (;; ++it) {
    // r = g - (A~ + L R) x
    if (df) apply_els_df(xo.p, xp.p, ro.p, rp.p, nrhs, s);
    else apply_els(xo.p, xp.p, ro.p, rp.p, nrhs, s);
    axpby(go.p, ro.p, ro.n, 1.0, -1.0, s);
    axpby(gp.p, rp.p, rp.n, 1.0, -1.0, s);
    std::vector<double> rn = col_dots(ro.p, rp.p, ro.p, rp.p, no, np, nrhs, 1, dots.p, s);
    worst = 0.0;
    for (int c = 0; c < nrhs; ++c) worst = std::max(worst, gn[c] > 0 ? std::sqrt(rn[c] / gn[c]) : 0.0);
    if (worst <= o.gmres_tol || it >= o.gmres_maxit) break;
    direct(ro.p, rp.p, dso.p, dsp.p);
    axpby(dso.p, xo.p, xo.n, 1.0, 1.0, s);
    axpby(dsp.p, xp.p, xp.n, 1.0, 1.0, s);
  }
  gather_scatter(xo.p, no, n_to_o.p, tau, 2 * Nn, n_from_o.p, nko, nrhs, s);
  gather_scatter(xp.p, np, n_to_p.p, tau, 2 * Nn, n_from_p.p, nkp, nrhs, s);
  *iters_out = it;
  *relres_out = worst;
}

void Refinement::solve_gmres(const double* g, double* tau, int nrhs, cudaStream_t s, int* iters_out,
                             double* relres_out, bool bf16, bool mixed) const {
  const Opts& o = wall->opts;
  // double-FP32 products only pay off once the right-hand sides fill the
  // GEMM tiles; below that the mixed mode is the FP32 mode
  mixed = mixed && nrhs > 8;
  auto op = [&](const double* xo_, const double* xp_, double* yo_, double* yp_) {
    if (mixed) apply_els_df(xo_, xp_, yo_, yp_, nrhs, s);
    else apply_els(xo_, xp_, yo_, yp_, nrhs, s);
  };
  TBuf<float> o32_in(mixed ? size_t(2 * No) * nrhs : 0, s), o32_out(mixed ? size_t(2 * No) * nrhs : 0, s);
  TBuf<float> p32_in(mixed ? size_t(2 * Np) * nrhs : 0, s), p32_out(mixed ? size_t(2 * Np) * nrhs : 0, s);
  // the operator with FP32 factors and vectors (relaxed iterations)
  auto op32 = [&](const double* xo_, const double* xp_, double* yo_, double* yp_) {
    k_d2f_v<<<g1(size_t(2 * No) * nrhs), 256, 0, s>>>(xo_, o32_in.p, size_t(2 * No) * nrhs);
    k_d2f_v<<<g1(size_t(2 * Np) * nrhs), 256, 0, s>>>(xp_, p32_in.p, size_t(2 * Np) * nrhs);
    RW_CHECK_LAUNCH();
    run_prog(els_prog32(s), o32_in.p, p32_in.p, o32_out.p, p32_out.p, (float*)nullptr, nrhs, s);
    k_f2d_v<<<g1(size_t(2 * No) * nrhs), 256, 0, s>>>(o32_out.p, yo_, size_t(2 * No) * nrhs);
    k_f2d_v<<<g1(size_t(2 * Np) * nrhs), 256, 0, s>>>(p32_out.p, yp_, size_t(2 * Np) * nrhs);
    RW_CHECK_LAUNCH();
  };
  require(wall->hbs.has_fp32 && hpp.has_fp32, "GMRES path: FP32 sweep data missing");
  require(!bf16 || (wall->hbs.has_bf16 && hpp.has_bf16), "GMRES path: BF16 sweep data missing");
  const int m = o.gmres_maxit;
  const int no = 2 * No, np = 2 * Np;
  // Krylov bases V (m+1 vectors) and Z (m vectors), o and p parts separately
  TBuf<double> Vo(size_t(no) * nrhs * (m + 1), s), Vp(size_t(np) * nrhs * (m + 1), s);
  TBuf<double> Zo(size_t(no) * nrhs * m, s), Zp(size_t(np) * nrhs * m, s);
  TBuf<double> xo(size_t(no) * nrhs, s), xp(size_t(np) * nrhs, s), ro(size_t(no) * nrhs, s), rp(size_t(np) * nrhs, s);
  TBuf<double> wo(size_t(no) * nrhs, s), wp(size_t(np) * nrhs, s), go(size_t(no) * nrhs, s), gp(size_t(np) * nrhs, s);
  TBuf<float> fo_in(size_t(no) * nrhs, s), fo_out(size_t(no) * nrhs, s), fp_in(size_t(np) * nrhs, s), fp_out(size_t(np) * nrhs, s);
  TBuf<double> dots(size_t(m + 1) * nrhs, s), coef(size_t(m + 1) * nrhs, s);
  // preconditioner's Woodbury vectors (mixed mode): r and z in FP32, in FP64
  TBuf<float> r32(mixed ? size_t(std::max(k, 1)) * nrhs : 0, s);
  TBuf<double> r64(mixed ? size_t(std::max(k, 1)) * nrhs : 0, s), z64(mixed ? size_t(std::max(k, 1)) * nrhs : 0, s);
  fill_zero(go.p, go.n, s);
  gather_scatter(g, 2 * Nn, n_from_o.p, go.p, no, n_to_o.p, nko, nrhs, s);
  gather_scatter(g, 2 * Nn, n_from_p.p, gp.p, np, n_to_p.p, nkp, nrhs, s);
  fill_zero(xo.p, xo.n, s);
  fill_zero(xp.p, xp.n, s);

  auto coldots = [&](const double* ao, const double* ap, const double* bo, const double* bp, int nb) {
    // dots[j * nrhs + c] = <a[:, c], b_j[:, c]>
    k_coldot2<<<dim3(nrhs, nb), 256, 0, s>>>(ao, bo, no, no, ap, bp, np, np, nrhs, dots.p);
    RW_CHECK_LAUNCH();
    std::vector<double> h(size_t(nb) * nrhs);
    RW_CUDA(cudaMemcpyAsync(h.data(), dots.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    RW_CUDA(cudaStreamSynchronize(s));
    return h;
  };
  auto comb = [&](double* yo, double* yp, const double* bo, const double* bp, int nb, const std::vector<double>& c) {
    RW_CUDA(cudaMemcpyAsync(coef.p, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    k_colcomb<<<dim3(g1(no), nrhs), 256, 0, s>>>(yo, bo, no, no, nrhs, nb, coef.p);
    k_colcomb<<<dim3(g1(np), nrhs), 256, 0, s>>>(yp, bp, np, np, nrhs, nb, coef.p);
    RW_CHECK_LAUNCH();
  };
  auto scale = [&](const double* xo_, const double* xp_, double* yo_, double* yp_, const std::vector<double>& c) {
    RW_CUDA(cudaMemcpyAsync(coef.p, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    k_colscale<<<dim3(g1(no), nrhs), 256, 0, s>>>(xo_, yo_, no, no, coef.p);
    k_colscale<<<dim3(g1(np), nrhs), 256, 0, s>>>(xp_, yp_, np, np, coef.p);
    RW_CHECK_LAUNCH();
  };
  auto precond = [&](const double* vo, const double* vp, double* zo, double* zp) {
    k_d2f_v<<<g1(size_t(no) * nrhs), 256, 0, s>>>(vo, fo_in.p, size_t(no) * nrhs);
    k_d2f_v<<<g1(size_t(np) * nrhs), 256, 0, s>>>(vp, fp_in.p, size_t(np) * nrhs);
    RW_CHECK_LAUNCH();
    if (mixed) {
      // sweeps and r = R y in one launch, z = W^{-1} r in FP64, y -= X z
      run_prog(pre_prog_a(bf16, s), fo_in.p, fp_in.p, fo_out.p, fp_out.p, r32.p, nrhs, s);
      if (k > 0) {
        k_f2d_v<<<g1(size_t(k) * nrhs), 256, 0, s>>>(r32.p, r64.p, size_t(k) * nrhs);
        RW_CHECK_LAUNCH();
        matvec<double>({GemvProb<double>{Winv.p, r64.p, z64.p, k, k, k, k, k, 1.0, 0.0}}, nrhs, s);
        k_d2f_v<<<g1(size_t(k) * nrhs), 256, 0, s>>>(z64.p, r32.p, size_t(k) * nrhs);
        RW_CHECK_LAUNCH();
        run_prog(pre_prog_b(s), (const float*)nullptr, (const float*)nullptr, fo_out.p, fp_out.p, r32.p, nrhs, s);
      }
    } else if (bf16) {
      wall->hbs.apply_inverse_bf16(fo_in.p, fo_out.p, nrhs, s);
      hpp.apply_inverse_bf16(fp_in.p, fp_out.p, nrhs, s);
    } else {
      wall->hbs.apply_inverse_f32(fo_in.p, fo_out.p, nrhs, s);
      hpp.apply_inverse_f32(fp_in.p, fp_out.p, nrhs, s);
    }
    k_f2d_v<<<g1(size_t(no) * nrhs), 256, 0, s>>>(fo_out.p, zo, size_t(no) * nrhs);
    k_f2d_v<<<g1(size_t(np) * nrhs), 256, 0, s>>>(fp_out.p, zp, size_t(np) * nrhs);
    RW_CHECK_LAUNCH();
    if (!mixed) woodbury_correct(zo, zp, nrhs, s);
  };

  std::vector<double> gnorm = coldots(go.p, gp.p, go.p, gp.p, 1);
  for (auto& v : gnorm) v = std::sqrt(v);
  int total_it = 0;
  double worst = 0.0;
  // Inexact (relaxed) products, mixed mode only (Bouras and Fraysse 2005,
  // Simoncini and Szyld 2003): once the residual estimate is below eta, the
  // error an operator product may carry without spoiling the final residual
  // grows as tol / residual, so the rest of the cycle uses the FP32 operator
  // (relative error ~3e-6, so eta = tol / 3e-6).  Each cycle starts from the
  // true residual with the accurate operator; a cycle whose true residual
  // still misses tol after a relaxed cycle runs without relaxation.
  bool relax = mixed;
  const double eta = o.gmres_tol / 3e-6;
  for (int cycle = 0;; ++cycle) {
    // r = g - A x (x = 0 in the first cycle: r = g)
    RW_CUDA(cudaMemcpyAsync(ro.p, go.p, go.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RW_CUDA(cudaMemcpyAsync(rp.p, gp.p, gp.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    std::vector<double> beta;
    if (cycle == 0) {
      beta = gnorm;
    } else {
      op(xo.p, xp.p, wo.p, wp.p);
      comb(ro.p, rp.p, wo.p, wp.p, 1, std::vector<double>(nrhs, -1.0));
      beta = coldots(ro.p, rp.p, ro.p, rp.p, 1);
      for (auto& v : beta) v = std::sqrt(v);
    }
    worst = 0.0;
    for (int c = 0; c < nrhs; ++c) worst = std::max(worst, gnorm[c] > 0 ? beta[c] / gnorm[c] : 0.0);
    if (worst <= o.gmres_tol || cycle == o.gmres_restarts) break;
    if (cycle > 0) relax = false;
    std::vector<double> inv(nrhs);
    for (int c = 0; c < nrhs; ++c) inv[c] = beta[c] > 0 ? 1.0 / beta[c] : 0.0;
    scale(ro.p, rp.p, Vo.p, Vp.p, inv);
    // Hessenberg and Givens data per column
    std::vector<std::vector<double>> H(nrhs, std::vector<double>(size_t(m + 1) * m, 0.0));
    std::vector<std::vector<double>> cs(nrhs, std::vector<double>(m)), sn(nrhs, std::vector<double>(m));
    std::vector<std::vector<double>> e(nrhs, std::vector<double>(m + 1, 0.0));
    for (int c = 0; c < nrhs; ++c) e[c][0] = beta[c];
    int j = 0;
    for (; j < m; ++j) {
      double* zoj = Zo.p + size_t(j) * no * nrhs;
      double* zpj = Zp.p + size_t(j) * np * nrhs;
      precond(Vo.p + size_t(j) * no * nrhs, Vp.p + size_t(j) * np * nrhs, zoj, zpj);
      if (relax && worst <= eta) op32(zoj, zpj, wo.p, wp.p);
      else op(zoj, zpj, wo.p, wp.p);
      // classical Gram-Schmidt, twice
      for (int pass = 0; pass < 2; ++pass) {
        std::vector<double> h = coldots(wo.p, wp.p, Vo.p, Vp.p, j + 1);
        std::vector<double> neg(h.size());
        for (size_t q = 0; q < h.size(); ++q) neg[q] = -h[q];
        comb(wo.p, wp.p, Vo.p, Vp.p, j + 1, neg);
        for (int c = 0; c < nrhs; ++c)
          for (int i = 0; i <= j; ++i) H[c][i + size_t(j) * (m + 1)] += h[size_t(i) * nrhs + c];
      }
      std::vector<double> hn = coldots(wo.p, wp.p, wo.p, wp.p, 1);
      std::vector<double> invn(nrhs);
      worst = 0.0;
      for (int c = 0; c < nrhs; ++c) {
        const double hnn = std::sqrt(hn[c]);
        H[c][j + 1 + size_t(j) * (m + 1)] = hnn;
        invn[c] = hnn > 0 ? 1.0 / hnn : 0.0;
        // apply previous rotations, then a new one
        double* col = &H[c][size_t(j) * (m + 1)];
        for (int i = 0; i < j; ++i) {
          const double t = cs[c][i] * col[i] + sn[c][i] * col[i + 1];
          col[i + 1] = -sn[c][i] * col[i] + cs[c][i] * col[i + 1];
          col[i] = t;
        }
        const double a = col[j], b = col[j + 1], r = std::hypot(a, b);
        cs[c][j] = r > 0 ? a / r : 1.0;
        sn[c][j] = r > 0 ? b / r : 0.0;
        col[j] = r;
        col[j + 1] = 0.0;
        e[c][j + 1] = -sn[c][j] * e[c][j];
        e[c][j] = cs[c][j] * e[c][j];
        worst = std::max(worst, gnorm[c] > 0 ? std::fabs(e[c][j + 1]) / gnorm[c] : 0.0);
      }
      scale(wo.p, wp.p, Vo.p + size_t(j + 1) * no * nrhs, Vp.p + size_t(j + 1) * np * nrhs, invn);
      ++total_it;
      if (worst <= 0.5 * o.gmres_tol) { ++j; break; }
    }
    // y = R^{-1} e per column, x += Z y
    std::vector<double> yc(size_t(j) * nrhs, 0.0);
    for (int c = 0; c < nrhs; ++c) {
      for (int i = j - 1; i >= 0; --i) {
        double acc = e[c][i];
        for (int l = i + 1; l < j; ++l) acc -= H[c][i + size_t(l) * (m + 1)] * yc[size_t(l) * nrhs + c];
        const double d = H[c][i + size_t(i) * (m + 1)];
        yc[size_t(i) * nrhs + c] = d != 0 ? acc / d : 0.0;
      }
    }
    if (j > 0) comb(xo.p, xp.p, Zo.p, Zp.p, j, yc);
  }
  // worst: the true relative residual of the last cycle start (the verified one)
  gather_scatter(xo.p, no, n_to_o.p, tau, 2 * Nn, n_from_o.p, nko, nrhs, s);
  gather_scatter(xp.p, np, n_to_p.p, tau, 2 * Nn, n_from_p.p, nkp, nrhs, s);
  *iters_out = total_it;
  *relres_out = worst;
}

}  // namespace rw
