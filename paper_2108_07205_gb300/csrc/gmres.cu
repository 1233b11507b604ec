// Mixed-precision path (Sec. 4.2): flexible GMRES in FP64 on the extended
// system (A~ + L R) tau_ext = g_ext (Eq. ELS_approximate), with A~ applied by
// the FP64 HBS forward representations of A_oo and A_pp and L R by the FP64
// factors.  The preconditioner is the Woodbury inverse of Sec. 4.2 whose
// A~^{-1} applications are HBS inverse sweeps in FP32 (or with the matrices
// in BF16, FP32 accumulation); X and W^{-1} stay FP64.
// Right preconditioning keeps the monitored residual equal to the true one.
// Every right-hand side runs its own Krylov space; the columns advance in
// lockstep and stop together once all have converged.
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

}  // namespace

void Refinement::solve_gmres(const double* g, double* tau, int nrhs, cudaStream_t s, int* iters_out,
                             double* relres_out, bool bf16) const {
  const Opts& o = wall->opts;
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
    if (bf16) {
      wall->hbs.apply_inverse_bf16(fo_in.p, fo_out.p, nrhs, s);
      hpp.apply_inverse_bf16(fp_in.p, fp_out.p, nrhs, s);
    } else {
      wall->hbs.apply_inverse_f32(fo_in.p, fo_out.p, nrhs, s);
      hpp.apply_inverse_f32(fp_in.p, fp_out.p, nrhs, s);
    }
    k_f2d_v<<<g1(size_t(no) * nrhs), 256, 0, s>>>(fo_out.p, zo, size_t(no) * nrhs);
    k_f2d_v<<<g1(size_t(np) * nrhs), 256, 0, s>>>(fp_out.p, zp, size_t(np) * nrhs);
    RW_CHECK_LAUNCH();
    woodbury_correct(zo, zp, nrhs, s);
  };

  std::vector<double> gnorm = coldots(go.p, gp.p, go.p, gp.p, 1);
  for (auto& v : gnorm) v = std::sqrt(v);
  int total_it = 0;
  double worst = 0.0;
  for (int cycle = 0; cycle < o.gmres_restarts; ++cycle) {
    // r = g - A x
    apply_els(xo.p, xp.p, wo.p, wp.p, nrhs, s);
    std::vector<double> minus1(nrhs, -1.0), one(nrhs, 1.0);
    RW_CUDA(cudaMemcpyAsync(ro.p, go.p, go.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RW_CUDA(cudaMemcpyAsync(rp.p, gp.p, gp.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    comb(ro.p, rp.p, wo.p, wp.p, 1, minus1);
    std::vector<double> beta = coldots(ro.p, rp.p, ro.p, rp.p, 1);
    worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
      beta[c] = std::sqrt(beta[c]);
      worst = std::max(worst, gnorm[c] > 0 ? beta[c] / gnorm[c] : 0.0);
    }
    if (worst <= o.gmres_tol) break;
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
      apply_els(zoj, zpj, wo.p, wp.p, nrhs, s);
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
  // final true residual
  apply_els(xo.p, xp.p, wo.p, wp.p, nrhs, s);
  RW_CUDA(cudaMemcpyAsync(ro.p, go.p, go.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  RW_CUDA(cudaMemcpyAsync(rp.p, gp.p, gp.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  comb(ro.p, rp.p, wo.p, wp.p, 1, std::vector<double>(nrhs, -1.0));
  std::vector<double> rn = coldots(ro.p, rp.p, ro.p, rp.p, 1);
  worst = 0.0;
  for (int c = 0; c < nrhs; ++c) worst = std::max(worst, gnorm[c] > 0 ? std::sqrt(rn[c]) / gnorm[c] : 0.0);
  gather_scatter(xo.p, no, n_to_o.p, tau, 2 * Nn, n_from_o.p, nko, nrhs, s);
  gather_scatter(xp.p, np, n_to_p.p, tau, 2 * Nn, n_from_p.p, nkp, nrhs, s);
  *iters_out = total_it;
  *relres_out = worst;
}

}  // namespace rw
