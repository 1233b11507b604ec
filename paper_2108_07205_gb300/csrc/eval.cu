// Geometry and kernel-matrix evaluation kernels (Sec. 2, Sec. 3.1, Sec. 3.3).
#include "eval.cuh"
#include "dense.cuh"
#include <algorithm>
#include <cmath>

namespace rw {

// ------------------------------------------------------------ quadrature
void gauss_legendre16(double* x, double* w) { gauss_legendre_n(16, x, w); }

void gauss_legendre_n(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    // Chebyshev-like initial guess, Newton on P_n via the three-term recurrence
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;  // ascending
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

namespace {

__constant__ double c_glx[16], c_glw[16];
// auxiliary 32-point rule of the hole matrix and the values l_j(u_f) of the
// 16-point Lagrange basis at its nodes (c_lag[f][j])
constexpr int kAux = 32;
__constant__ double c_ux[kAux], c_uw[kAux], c_lag[kAux][16];
// (n + 1/2) P_n(u_f): the Legendre factors of the product weights Lam_f
__constant__ double c_pn[kAux][kAux];

struct Pt { double x, y, dx, dy, ddx, ddy; };

__device__ Pt curve_eval(const Curve& c, double t) {
  Pt q;
  if (c.kind == RW_CURVE_STAR || c.kind == kCurveHole) {
    const double a = c.p[0], k = c.p[1], sc = c.p[2];
    double ct, st, ck, sk;
    sincos(t, &st, &ct);
    sincos(k * t, &sk, &ck);
    const double r = sc * (1.0 + a * ck), r1 = -sc * a * k * sk, r2 = -sc * a * k * k * ck;
    q.x = r * ct; q.y = r * st;
    q.dx = r1 * ct - r * st; q.dy = r1 * st + r * ct;
    q.ddx = r2 * ct - 2.0 * r1 * st - r * ct;
    q.ddy = r2 * st + 2.0 * r1 * ct - r * st;
    if (c.kind == kCurveHole) { q.x += c.p[3]; q.y += c.p[4]; }
  } else {
    // superellipse (A cos t, B sin t) (cos^p + sin^p)^(-1/p), y squeezed by
    // q(x) = 1 - delta (1 + cos(pi x / A)) / 2
    const double A = c.p[0], B = c.p[1], p = c.p[2], delta = c.p[3];
    double ct, st;
    sincos(t, &st, &ct);
    const double cp = pow(ct, p), sp = pow(st, p);
    const double cp1 = pow(ct, p - 1.0), sp1 = pow(st, p - 1.0);
    const double cp2 = pow(ct, p - 2.0), sp2 = pow(st, p - 2.0);
    const double h = cp + sp;
    const double h1 = p * (-cp1 * st + sp1 * ct);
    const double h2 = p * ((p - 1.0) * cp2 * st * st - cp + (p - 1.0) * sp2 * ct * ct - sp);
    const double sg = pow(h, -1.0 / p);
    const double sg1 = -(1.0 / p) * sg / h * h1;
    const double sg2 = -(1.0 / p) * ((-1.0 / p - 1.0) * sg / (h * h) * h1 * h1 + sg / h * h2);
    const double X = A * ct * sg, X1 = A * (-st * sg + ct * sg1), X2 = A * (-ct * sg - 2.0 * st * sg1 + ct * sg2);
    const double Y = B * st * sg, Y1 = B * (ct * sg + st * sg1), Y2 = B * (-st * sg + 2.0 * ct * sg1 + st * sg2);
    double sx, cx;
    sincos(kPi * X / A, &sx, &cx);
    const double qv = 1.0 - 0.5 * delta * (1.0 + cx);
    const double qx = 0.5 * delta * (kPi / A) * sx;
    const double qxx = 0.5 * delta * (kPi / A) * (kPi / A) * cx;
    const double Q1 = qx * X1, Q2 = qxx * X1 * X1 + qx * X2;
    q.x = X; q.dx = X1; q.ddx = X2;
    q.y = Y * qv; q.dy = Y1 * qv + Y * Q1; q.ddy = Y2 * qv + 2.0 * Y1 * Q1 + Y * Q2;
  }
  return q;
}

__global__ void k_nodes(Curve c, const double* ta, const double* tb, int n_int, double* out, int ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 16 * n_int) return;
  const int pnl = i / 16, q = i % 16;
  const double a = ta[pnl], b = tb[pnl];
  const double half = 0.5 * (b - a), mid = 0.5 * (b + a);
  const double t = mid + half * c_glx[q];
  const Pt g = curve_eval(c, t);
  const double sp = sqrt(g.dx * g.dx + g.dy * g.dy);
  out[i] = g.x;
  out[i + ld] = g.y;
  out[i + 2 * size_t(ld)] = g.dy / sp;
  out[i + 3 * size_t(ld)] = -g.dx / sp;
  out[i + 4 * size_t(ld)] = c_glw[q] * half * sp;
  out[i + 5 * size_t(ld)] = (g.dx * g.ddy - g.dy * g.ddx) / (sp * sp * sp);
}

// Moments M_n(t) = int_{-1}^{1} P_n(s) log|t - s| ds, n = 0..NM-1, of the
// Legendre polynomials against the logarithm.  Integration by parts with
// P_n = (P_{n+1}' - P_{n-1}') / (2n + 1) gives M_n = 2 (Q_{n+1}(t) -
// Q_{n-1}(t)) / (2n + 1), where Q_m(t) = (1/2) int P_m(s) / (t - s) ds (a
// principal value for |t| < 1) obeys the Legendre three-term recurrence from
// Q_0 = (1/2) log|(1 + t) / (1 - t)|, Q_1 = t Q_0 - 1.  For |t| < 1 the
// recurrence runs forward; for |t| > 1, where Q_m is the recurrence's
// minimal solution, it runs backward from a start index past which the
// neglected dominant part is below rounding (Miller's algorithm) and is
// normalised by Q_0.  M_0 is the elementary integral.
template <int NM>
__device__ void log_moments(double t, double* M) {
  double Q[NM + 1];
  const double at = fabs(t);
  if (at < 1.0) {
    Q[0] = 0.5 * log((1.0 + t) / (1.0 - t));
    Q[1] = t * Q[0] - 1.0;
    for (int n = 1; n < NM; ++n) Q[n + 1] = ((2.0 * n + 1.0) * t * Q[n] - n * Q[n - 1]) / (n + 1.0);
  } else {
    const double rho = at + sqrt((at - 1.0) * (at + 1.0));
    const int n0 = min(NM + 1 + int(ceil(40.0 / log(rho))), 20000);
    double qn1 = 0.0, qn = 1.0;  // Q_{n+1}, Q_n up to a common factor
    for (int n = n0; n >= 1; --n) {
      const double qm = ((2.0 * n + 1.0) * t * qn - (n + 1.0) * qn1) / n;
      qn1 = qn;
      qn = qm;
      if (n - 1 <= NM) Q[n - 1] = qn;
      if (fabs(qn) > 1e200) {
        qn *= 1e-200;
        qn1 *= 1e-200;
        for (int m = max(n - 1, 0); m <= NM; ++m) Q[m] *= 1e-200;
      }
    }
    const double sc = 0.5 * log((t + 1.0) / (t - 1.0)) / Q[0];
    for (int m = 0; m <= NM; ++m) Q[m] *= sc;
  }
  M[0] = (t + 1.0) * log(fabs(t + 1.0)) - (t - 1.0) * log(fabs(t - 1.0)) - 2.0;
  for (int n = 1; n < NM; ++n) M[n] = 2.0 * (Q[n + 1] - Q[n - 1]) / (2.0 * n + 1.0);
}

// The 2 x 2 block of A between a target point t and a source point s
// (A(t a, s b) for a, b in {0, 1}): one distance, one division.
struct Blk2 { double v[2][2]; };
__device__ __forceinline__ Blk2 a_block(const NodesView& T, int t, const NodesView& Sv, int s, bool same_point) {
  Blk2 o;
  const double ws = Sv.w[s];
  if (T.kind | Sv.kind) {
    // a hole is involved (App. B): combined field of a hole source, double
    // layer of a wall source at a hole point; never the same point
    const double rx = T.x[t] - Sv.x[s], ry = T.y[t] - Sv.y[s];
    const double r2 = rx * rx + ry * ry, inv = 1.0 / r2;
    const double fac = ws * (rx * Sv.nx[s] + ry * Sv.ny[s]) * inv * inv * (1.0 / kPi);
    const double sl = Sv.kind ? ws * (0.25 / kPi) : 0.0, lg = Sv.kind ? -0.5 * log(r2) : 0.0;
    const double r[2] = {rx, ry};
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) o.v[a][b] = fac * r[a] * r[b] + sl * ((a == b ? lg : 0.0) + r[a] * r[b] * inv);
    return o;
  }
  const double ntx = T.nx[t], nty = T.ny[t], nsx = Sv.nx[s], nsy = Sv.ny[s];
  const double nt[2] = {ntx, nty}, ns[2] = {nsx, nsy};
  if (same_point) {
    const double ta[2] = {-nty, ntx};
    const double kap = T.kappa[t] * ws * (0.5 / kPi);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) o.v[a][b] = nt[a] * ns[b] * ws - kap * ta[a] * ta[b] - (a == b ? 0.5 : 0.0);
  } else {
    const double rx = T.x[t] - Sv.x[s], ry = T.y[t] - Sv.y[s];
    const double inv = 1.0 / (rx * rx + ry * ry);
    const double fac = ws * (rx * nsx + ry * nsy) * inv * inv * (1.0 / kPi);
    const double r[2] = {rx, ry};
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) o.v[a][b] = nt[a] * ns[b] * ws + fac * r[a] * r[b];
  }
  return o;
}

// Entry of A = -1/2 I + D + N (Sec. 2, Remark 2.1) for row DOF (i, a) of node
// set R and column DOF (j, b) of node set C.  same_set marks R == C, where
// i == j gives the diagonal block -1/2 I - (kappa_i w_i / 2 pi) t t^T
// + w_i n_i n_i^T (the smooth limit of the double layer on the curve).
// With holes (App. B): a hole source (C.kind 1) contributes its combined
// field w_j (D + S)(x_i, y_j) and a wall source seen at a hole point (R.kind
// 1) its double layer w_j D(x_i, y_j), neither with the N term.  Pairs on
// one hole are not evaluated here (their single layer needs the singular
// rule of the hole matrix).
__device__ __forceinline__ double a_entry(const NodesView& R, int i, int a,
                                          const NodesView& C, int j, int b,
                                          bool same_set) {
  const double wj = C.w[j];
  if (C.kind | R.kind) {
    const double rx = R.x[i] - C.x[j], ry = R.y[i] - C.y[j];
    const double r2 = rx * rx + ry * ry, inv = 1.0 / r2;
    const double ra = a ? ry : rx, rb = b ? ry : rx;
    double val = wj * (rx * C.nx[j] + ry * C.ny[j]) * inv * inv * (1.0 / kPi) * ra * rb;
    if (C.kind) val += wj * (0.25 / kPi) * ((a == b ? -0.5 * log(r2) : 0.0) + ra * rb * inv);
    return val;
  }
  const double nia = a ? R.ny[i] : R.nx[i];
  const double njb = b ? C.ny[j] : C.nx[j];
  double val = nia * njb * wj;
  if (same_set && i == j) {
    const double ta = a ? R.nx[i] : -R.ny[i];
    const double tb = b ? R.nx[i] : -R.ny[i];
    val -= R.kappa[i] * wj * (0.5 / kPi) * ta * tb;
    if (a == b) val -= 0.5;
  } else {
    const double rx = R.x[i] - C.x[j], ry = R.y[i] - C.y[j];
    const double r2 = rx * rx + ry * ry;
    const double rdn = rx * C.nx[j] + ry * C.ny[j];
    const double fac = wj * rdn / (kPi * r2 * r2);
    val += fac * (a ? ry : rx) * (b ? ry : rx);
  }
  return val;
}

// Single layer of one exterior-wall pair (Sec. 2.2) whose target x_i sits
// within kExtNear half-widths of the source's panel (midpoint tm, half-width
// th in t, local coordinate loc of the target; source node q of the panel):
// the density's degree-15 interpolant on the panel against the exact kernel,
// with the geometry exact -- Legendre product integration of the logarithm
// (generalised Gaussian corrections in the sense of Sec. 5, exact for the
// interpolant) on a 32-point auxiliary rule (u_f, nu_f):
//   int log|x_i - y(s)| l_q(s) |y'(s)| th ds
//     ~ th sum_f [Lam_f(loc) + nu_f phi(u_f)] |y'(u_f)| l_q(u_f),
//   Lam_f(loc) = nu_f sum_{n<32} (2n+1)/2 P_n(u_f) M_n(loc),
//   phi(s) = log|x_i - y(s)| - log|loc - s|  (smooth),
// and r r^T / |r|^2 by the auxiliary rule alone (it is smooth along the
// curve).  out = w_j S(x_i, y_j) entries (xx, xy, yy).
__device__ __noinline__ void ext_near_sl(double xi, double yi, double loc, const Curve& c, double tm, double th,
                                         int q, double* out) {
  double M[kAux];
  log_moments<kAux>(loc, M);
  double sl = 0.0, sxx = 0.0, sxy = 0.0, syy = 0.0;
  for (int f = 0; f < kAux; ++f) {
    const double u = c_ux[f];
    double acc = 0.0;
#pragma unroll 8
    for (int n = 0; n < kAux; ++n) acc += c_pn[f][n] * M[n];
    const Pt g = curve_eval(c, tm + th * u);
    const double gl = sqrt(g.dx * g.dx + g.dy * g.dy) * c_lag[f][q];
    const double rx = xi - g.x, ry = yi - g.y, r2 = rx * rx + ry * ry;
    const double phi = 0.5 * log(r2 / ((loc - u) * (loc - u)));
    sl += c_uw[f] * (acc + phi) * gl;
    const double wg = c_uw[f] * gl / r2;
    sxx += wg * rx * rx;
    sxy += wg * rx * ry;
    syy += wg * ry * ry;
  }
  const double c4 = 0.25 / kPi;
  out[0] = c4 * th * (sxx - sl);
  out[1] = c4 * th * sxy;
  out[2] = c4 * th * (syy - sl);
}

// The 2 x 2 block of 1/2 I + D + S (Eq. exterior_BIE) between a target t and
// a source s of exterior-wall node sets (same_point: t and s are one node).
// The double layer takes the plain panel rule with the curvature limit at
// the same point; the single layer the plain rule, or ext_near_sl where the
// target is near the source's panel.
__device__ Blk2 a_block_ext(const NodesView& T, int t, const NodesView& Sv, int s, bool same_point) {
  Blk2 o;
  const double ws = Sv.w[s];
  const double rx = T.x[t] - Sv.x[s], ry = T.y[t] - Sv.y[s];
  const double r[2] = {rx, ry};
  if (same_point) {
    const double ta[2] = {-T.ny[t], T.nx[t]};
    const double kap = -T.kappa[t] * ws * (0.5 / kPi);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) o.v[a][b] = kap * ta[a] * ta[b] + (a == b ? 0.5 : 0.0);
  } else {
    const double inv = 1.0 / (rx * rx + ry * ry);
    const double fac = ws * (rx * Sv.nx[s] + ry * Sv.ny[s]) * inv * inv * (1.0 / kPi);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) o.v[a][b] = fac * r[a] * r[b];
  }
  const double loc = ext_loc(T.t[t], Sv.tm[s], Sv.th[s]);
  if (fabs(loc) < kExtNear) {
    double sl[3];
    ext_near_sl(T.x[t], T.y[t], same_point ? c_glx[s & 15] : loc, Sv.curve, Sv.tm[s], Sv.th[s], s & 15, sl);
    o.v[0][0] += sl[0];
    o.v[0][1] += sl[1];
    o.v[1][0] += sl[1];
    o.v[1][1] += sl[2];
  } else {
    const double r2 = rx * rx + ry * ry, inv = 1.0 / r2, lg = -0.5 * log(r2), c = ws * (0.25 / kPi);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) o.v[a][b] += c * ((a == b ? lg : 0.0) + r[a] * r[b] * inv);
  }
  return o;
}

template <bool EXT>
__device__ __forceinline__ Blk2 block_of(const NodesView& T, int t, const NodesView& Sv, int s, bool same_point) {
  if constexpr (EXT) return a_block_ext(T, t, Sv, s, same_point);
  else return a_block(T, t, Sv, s, same_point);
}
template <bool EXT>
__device__ __forceinline__ double entry_of(const NodesView& R, int i, int a, const NodesView& C, int j, int b,
                                           bool same_set) {
  if constexpr (EXT) return a_block_ext(R, i, C, j, same_set && i == j).v[a][b];
  else return a_entry(R, i, a, C, j, b, same_set);
}

// Feature list section (entries of A against the DOFs e[0..n)): pairs of
// consecutive entries that are the two components of one point share one
// 2 x 2 block evaluation.
template <bool EXT>
__device__ __forceinline__ void idmat_section(const IdMatProb& P, double* Wc, int ip, int ia, const NodesView& S,
                                              const int* e, int n, const NodesView& E, bool es) {
  for (int cp = threadIdx.x; 2 * cp < n; cp += blockDim.x) {
    const int c = 2 * cp;
    const int e0 = e[c];
    const bool pair = c + 1 < n && (e0 & 1) == 0 && e[c + 1] == e0 + 1;
    if (pair) {
      const int j = e0 >> 1;
      const bool same = es && j == ip;
      if (P.kind == 0) {
        const Blk2 B = block_of<EXT>(S, ip, E, j, same);
        Wc[c] = B.v[ia][0];
        Wc[c + 1] = B.v[ia][1];
      } else {
        const Blk2 B = block_of<EXT>(E, j, S, ip, same);
        Wc[c] = B.v[0][ia];
        Wc[c + 1] = B.v[1][ia];
      }
    } else {
      for (int q = c; q < min(n, c + 2); ++q) {
        const int eq = e[q];
        Wc[q] = P.kind == 0 ? entry_of<EXT>(S, ip, ia, E, eq >> 1, eq & 1, es)
                            : entry_of<EXT>(E, eq >> 1, eq & 1, S, ip, ia, es);
      }
    }
  }
}

// Rows of W (features) for the candidates of one problem per blockIdx.y:
// near-field sections, then the proxy section (points tabulated once per
// block; one distance, one division and at most one logarithm per proxy
// point), then the normal column.
template <bool EXT>
__global__ void k_idmat(const IdMatProb* probs, int max_M, NodesView S, NodesView E1, bool e1s, NodesView E2,
                        bool e2s) {
  const IdMatProb P = probs[blockIdx.y];
  extern __shared__ double ztab[];  // 4 x max_M
  double* zx = ztab;
  double* zy = ztab + max_M;
  double* zc = ztab + 2 * max_M;
  double* zs = ztab + 3 * max_M;
  const int M = P.M * (P.ncirc > 1 ? P.ncirc : 1);
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    const int c = q / P.M, qq = q - c * P.M;
    const double ccx = P.ncirc > 1 ? P.circ[3 * c] : P.cx;
    const double ccy = P.ncirc > 1 ? P.circ[3 * c + 1] : P.cy;
    const double cR = P.ncirc > 1 ? P.circ[3 * c + 2] : P.R;
    double sn, cs;
    sincospi(2.0 * qq / P.M, &sn, &cs);
    zx[q] = ccx + cR * cs;
    zy[q] = ccy + cR * sn;
    zc[q] = cs;
    zs[q] = sn;
  }
  __syncthreads();
  const int base = P.n1 + P.n2;
  for (int i = blockIdx.x; i < P.m; i += gridDim.x) {
    double* Wc = P.W + size_t(i) * P.ldw;
    const int d = P.cand[i];
    const int ip = d >> 1, ia = d & 1;
    idmat_section<EXT>(P, Wc, ip, ia, S, P.e1, P.n1, E1, e1s);
    idmat_section<EXT>(P, Wc + P.n1, ip, ia, S, P.e2, P.n2, E2, e2s);
    const double xi = S.x[ip], yi = S.y[ip];
    if (P.kind == 0) {
      // field at x_i of unit sources at z_q: Stokeslet (columns 4q, 4q+1)
      // and double layer with the circle's outward normal (4q+2, 4q+3)
      for (int q = threadIdx.x; q < M; q += blockDim.x) {
        const double rx = xi - zx[q], ry = yi - zy[q], r2 = rx * rx + ry * ry;
        const double inv = 1.0 / r2, lg = -0.5 * log(r2), ra = ia ? ry : rx;
        const double f = (rx * zc[q] + ry * zs[q]) * inv * inv * (1.0 / kPi);
        double* w = Wc + base + 4 * q;
        w[0] = (1.0 / (4.0 * kPi)) * ((ia == 0 ? lg : 0.0) + ra * rx * inv);
        w[1] = (1.0 / (4.0 * kPi)) * ((ia == 1 ? lg : 0.0) + ra * ry * inv);
        w[2] = ra * rx * f;
        w[3] = ra * ry * f;
      }
    } else {
      // field at z_q (components 2q, 2q+1) of a unit density at x_i
      const double nxi = S.nx[ip], nyi = S.ny[ip], wi = S.w[ip];
      for (int q = threadIdx.x; q < M; q += blockDim.x) {
        const double rx = zx[q] - xi, ry = zy[q] - yi;
        const double inv = 1.0 / (rx * rx + ry * ry);
        const double fac = wi * (rx * nxi + ry * nyi) * inv * inv * (1.0 / kPi) * (ia ? ry : rx);
        Wc[base + 2 * q] = fac * rx;
        Wc[base + 2 * q + 1] = fac * ry;
        if (EXT && P.sl_in) {
          // single layer of the combined field: w_i S(z_q, x_i) e_ia
          const double c = wi * (0.25 / kPi), lg = -0.5 * log(rx * rx + ry * ry), ra = ia ? ry : rx;
          Wc[base + 2 * M + 2 * q] = c * ((ia == 0 ? lg : 0.0) + rx * ra * inv);
          Wc[base + 2 * M + 2 * q + 1] = c * ((ia == 1 ? lg : 0.0) + ry * ra * inv);
        }
      }
    }
    if (P.normal && threadIdx.x == 0) {
      const double n = ia ? S.ny[ip] : S.nx[ip];
      Wc[P.ncol - 1] = P.kind == 0 ? n : n * S.w[ip];
    }
  }
}

// ext_near_sl for all 16 source nodes of one panel at once: the moments, the
// curve at the auxiliary nodes and the logarithms are shared by the 16, only
// the Lagrange factor differs.  out[3 q + (0, 1, 2)] = entries xx, xy, yy of
// w_j S(x_i, y_j) for source node q.
__device__ __noinline__ void ext_near_sl_panel(double xi, double yi, double loc, const Curve& c, double tm, double th,
                                               double* out) {
  double M[kAux];
  log_moments<kAux>(loc, M);
  double sl[16], sxx[16], sxy[16], syy[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) sl[q] = sxx[q] = sxy[q] = syy[q] = 0.0;
  for (int f = 0; f < kAux; ++f) {
    const double u = c_ux[f];
    double acc = 0.0;
#pragma unroll 8
    for (int n = 0; n < kAux; ++n) acc += c_pn[f][n] * M[n];
    const Pt g = curve_eval(c, tm + th * u);
    const double sp = sqrt(g.dx * g.dx + g.dy * g.dy);
    const double rx = xi - g.x, ry = yi - g.y, r2 = rx * rx + ry * ry;
    const double phi = 0.5 * log(r2 / ((loc - u) * (loc - u)));
    const double bl = c_uw[f] * (acc + phi) * sp, bt = c_uw[f] * sp / r2;
    const double txx = bt * rx * rx, txy = bt * rx * ry, tyy = bt * ry * ry;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const double lq = c_lag[f][q];
      sl[q] += bl * lq;
      sxx[q] += txx * lq;
      sxy[q] += txy * lq;
      syy[q] += tyy * lq;
    }
  }
  const double c4 = 0.25 / kPi;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    out[3 * q] = c4 * th * (sxx[q] - sl[q]);
    out[3 * q + 1] = c4 * th * sxy[q];
    out[3 * q + 2] = c4 * th * (syy[q] - sl[q]);
  }
}

// Exterior walls, blocks with contiguous rows and columns: one CTA per source
// panel (16 points = 32 columns), one thread per target point.  A target near
// the panel forms the singular rule's weights for all 16 source nodes once
// (ext_near_sl_panel); the double layer and the plain single layer per pair.
__global__ void k_blocks_ext_panels(const BlockProb* probs, NodesView s0, NodesView s1) {
  const BlockProb P = probs[blockIdx.y];
  const NodesView& R = P.rset ? s1 : s0;
  const NodesView& C = P.cset ? s1 : s0;
  const bool same = P.rset == P.cset;
  const int pc0 = P.c0 / 32, pc1 = (P.c0 + P.mc - 1) / 32;   // column panels
  const int i0 = P.r0 / 2, i1 = (P.r0 + P.mr - 1) / 2;       // target points
  for (int pc = pc0 + blockIdx.x; pc <= pc1; pc += gridDim.x) {
    const int j0 = 16 * pc;
    const double tm = C.tm[j0], th = C.th[j0];
    for (int i = i0 + threadIdx.x; i <= i1; i += blockDim.x) {
      const double loc = ext_loc(R.t[i], tm, th);
      const bool near = fabs(loc) < kExtNear;
      const bool own = same && (i >> 4) == pc;
      double w[48];
      if (near) ext_near_sl_panel(R.x[i], R.y[i], own ? c_glx[i & 15] : loc, C.curve, tm, th, w);
      for (int q = 0; q < 16; ++q) {
        const int j = j0 + q;
        if (2 * j + 1 < P.c0 || 2 * j >= P.c0 + P.mc) continue;
        const double ws = C.w[j];
        const double rx = R.x[i] - C.x[j], ry = R.y[i] - C.y[j];
        const double r[2] = {rx, ry};
        double b[2][2];
        if (same && i == j) {
          const double ta[2] = {-R.ny[i], R.nx[i]};
          const double kap = -R.kappa[i] * ws * (0.5 / kPi);
          for (int a = 0; a < 2; ++a)
            for (int e = 0; e < 2; ++e) b[a][e] = kap * ta[a] * ta[e] + (a == e ? 0.5 : 0.0);
        } else {
          const double inv = 1.0 / (rx * rx + ry * ry);
          const double fac = ws * (rx * C.nx[j] + ry * C.ny[j]) * inv * inv * (1.0 / kPi);
          for (int a = 0; a < 2; ++a)
            for (int e = 0; e < 2; ++e) b[a][e] = fac * r[a] * r[e];
        }
        if (near) {
          b[0][0] += w[3 * q];
          b[0][1] += w[3 * q + 1];
          b[1][0] += w[3 * q + 1];
          b[1][1] += w[3 * q + 2];
        } else {
          const double r2 = rx * rx + ry * ry, inv = 1.0 / r2, lg = -0.5 * log(r2), cc = ws * (0.25 / kPi);
          for (int a = 0; a < 2; ++a)
            for (int e = 0; e < 2; ++e) b[a][e] += cc * ((a == e ? lg : 0.0) + r[a] * r[e] * inv);
        }
        for (int a = 0; a < 2; ++a) {
          const int row = 2 * i + a - P.r0;
          if (row < 0 || row >= P.mr) continue;
          for (int e = 0; e < 2; ++e) {
            const int col = 2 * j + e - P.c0;
            if (col < 0 || col >= P.mc) continue;
            P.out[row + size_t(col) * P.ld] = P.scale * b[a][e];
          }
        }
      }
    }
  }
}

// Exterior walls: a thread forms the whole 2 x 2 block of a point pair once
// (the singular rule's weights are the expensive part) and writes the four
// entries when the problem's rows and columns come in (2i, 2i + 1) pairs;
// other entries one by one.
__global__ void k_blocks_ext(const BlockProb* probs, NodesView s0, NodesView s1) {
  const BlockProb P = probs[blockIdx.y];
  const NodesView& R = P.rset ? s1 : s0;
  const NodesView& C = P.cset ? s1 : s0;
  const bool same = P.rset == P.cset;
  for (int c = 2 * blockIdx.x; c < P.mc; c += 2 * gridDim.x) {
    const int c1 = min(c + 2, P.mc);
    const int dc0 = P.cols ? P.cols[c] : P.c0 + c;
    const bool cp = c1 - c == 2 && (dc0 & 1) == 0 && (P.cols ? P.cols[c + 1] : P.c0 + c + 1) == dc0 + 1;
    for (int r = 2 * threadIdx.x; r < P.mr; r += 2 * blockDim.x) {
      const int r1 = min(r + 2, P.mr);
      const int dr0 = P.rows ? P.rows[r] : P.r0 + r;
      const bool rp = r1 - r == 2 && (dr0 & 1) == 0 && (P.rows ? P.rows[r + 1] : P.r0 + r + 1) == dr0 + 1;
      if (rp && cp) {
        const int i = dr0 >> 1, j = dc0 >> 1;
        const Blk2 B = a_block_ext(R, i, C, j, same && i == j);
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) P.out[(r + a) + size_t(c + b) * P.ld] = P.scale * B.v[a][b];
      } else {
        for (int rr = r; rr < r1; ++rr)
          for (int cc = c; cc < c1; ++cc) {
            const int dr = P.rows ? P.rows[rr] : P.r0 + rr;
            const int dc = P.cols ? P.cols[cc] : P.c0 + cc;
            P.out[rr + size_t(cc) * P.ld] = P.scale * entry_of<true>(R, dr >> 1, dr & 1, C, dc >> 1, dc & 1, same);
          }
      }
    }
  }
}

template <bool EXT>
__global__ void k_blocks(const BlockProb* probs, NodesView s0, NodesView s1) {
  const BlockProb P = probs[blockIdx.y];
  const NodesView& R = P.rset ? s1 : s0;
  const NodesView& C = P.cset ? s1 : s0;
  const bool same = P.rset == P.cset;
  for (int c = blockIdx.x; c < P.mc; c += gridDim.x) {
    const int dc = P.cols ? P.cols[c] : P.c0 + c;
    for (int r = threadIdx.x; r < P.mr; r += blockDim.x) {
      const int dr = P.rows ? P.rows[r] : P.r0 + r;
      P.out[r + size_t(c) * P.ld] = P.scale * entry_of<EXT>(R, dr >> 1, dr & 1, C, dc >> 1, dc & 1, same);
    }
  }
}

__global__ void k_transpose(const TransProb* probs) {
  const TransProb P = probs[blockIdx.y];
  for (int j = blockIdx.x; j < P.m; j += gridDim.x)  // out(i, j) = in(j, i)
    for (int i = threadIdx.x; i < P.n; i += blockDim.x) P.out[i + size_t(j) * P.ldo] = P.in[j + size_t(i) * P.ldi];
}

__global__ void k_copy(const CopyProb* probs) {
  const CopyProb P = probs[blockIdx.y];
  for (int j = blockIdx.x; j < P.n; j += gridDim.x)
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) P.out[i + size_t(j) * P.ldo] = P.in[i + size_t(j) * P.ldi];
}

// One CTA per (target, group of up to kVelRhs right-hand sides); sources
// split over the threads.  The geometric factors of a (target, source) pair
// are formed once and applied to every right-hand side of the group.  Wall
// sources carry the double layer; hole sources (kind 1) the combined field,
// whose single layer adds w_j S(x, y_j) tau_j.
// The sources may be cut into gridDim.z chunks (chunks != null): each
// chunk's sums go to chunks[z] and k_velocity_sum adds them in order.
constexpr int kVelRhs = 8;
__global__ void __launch_bounds__(256) k_velocity(NodesView nd, const double* tau, int ldt, int nt, int nrhs,
                                                  const double* tg, double* u, int acc, double* chunks) {
  const int t = blockIdx.x, r0 = blockIdx.y * kVelRhs, nr = min(kVelRhs, nrhs - r0);
  const int per = (nd.n + gridDim.z - 1) / gridDim.z, j0 = blockIdx.z * per, j1 = min(nd.n, j0 + per);
  const double x = tg[2 * t], y = tg[2 * t + 1];
  double ux[kVelRhs], uy[kVelRhs];
#pragma unroll
  for (int q = 0; q < kVelRhs; ++q) ux[q] = uy[q] = 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const double rx = x - nd.x[j], ry = y - nd.y[j], r2 = rx * rx + ry * ry, inv = 1.0 / r2;
    const double fac = nd.w[j] * (rx * nd.nx[j] + ry * nd.ny[j]) * inv * inv * (1.0 / kPi);
    const double c = nd.kind ? nd.w[j] * (0.25 / kPi) : 0.0, lg = nd.kind ? -0.5 * log(r2) : 0.0;
#pragma unroll
    for (int q = 0; q < kVelRhs; ++q) {
      if (q >= nr) break;
      const double* tr = tau + size_t(r0 + q) * ldt;
      const double tx = tr[2 * j], ty = tr[2 * j + 1];
      const double rt = rx * tx + ry * ty;
      ux[q] += fac * rx * rt;
      uy[q] += fac * ry * rt;
      if (nd.kind) {
        const double qq = rt * inv;
        ux[q] += c * (lg * tx + rx * qq);
        uy[q] += c * (lg * ty + ry * qq);
      }
    }
  }
  // block sums in a fixed order: warps by shuffles, then warp 0 over warps
  __shared__ double part[2 * kVelRhs][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < kVelRhs; ++q) {
    double a = ux[q], b = uy[q];
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, off);
      b += __shfl_down_sync(0xffffffffu, b, off);
    }
    if (lane == 0) { part[2 * q][warp] = a; part[2 * q + 1][warp] = b; }
  }
  __syncthreads();
  if (warp == 0) {
    for (int v = 0; v < 2 * nr; ++v) {
      double a = lane < nw ? part[v][lane] : 0.0;
      for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
      if (lane == 0) {
        const size_t o = size_t(r0 + v / 2) * 2 * nt + 2 * t + (v & 1);
        if (chunks) {
          chunks[size_t(blockIdx.z) * nrhs * 2 * nt + o] = a;
        } else {
          double* ur = u + o;
          *ur = (acc ? *ur : 0.0) + a;
        }
      }
    }
  }
}

__global__ void k_velocity_sum(const double* part, int nchunk, size_t n, double* u, int acc) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    double a = 0.0;
    for (int z = 0; z < nchunk; ++z) a += part[size_t(z) * n + i];
    u[i] = (acc ? u[i] : 0.0) + a;
  }
}

// Pressure of the double-layer velocity (Sec. 2): p(x) = sum_j w_j P(x, y_j)
// . tau_j, P_j = (1/pi)(-n_j / r^2 + 2 r_j (r . n) / r^4), mu = 1; hole
// sources (kind 1) add the single layer's pressure w_j (r . tau_j) / (2 pi
// r^2).  One CTA per (target, right-hand side), sources split over threads.
__global__ void k_pressure(NodesView nd, const double* tau, int ldt, int nt, const double* tg, double* p, int acc) {
  const int t = blockIdx.x, r = blockIdx.y;
  const double x = tg[2 * t], y = tg[2 * t + 1];
  const double* tr = tau + size_t(r) * ldt;
  double dl = 0.0, sl = 0.0;
  for (int j = threadIdx.x; j < nd.n; j += blockDim.x) {
    const double rx = x - nd.x[j], ry = y - nd.y[j];
    const double inv = 1.0 / (rx * rx + ry * ry);
    const double ndt = nd.nx[j] * tr[2 * j] + nd.ny[j] * tr[2 * j + 1];
    const double rdt = rx * tr[2 * j] + ry * tr[2 * j + 1];
    const double rdn = rx * nd.nx[j] + ry * nd.ny[j];
    dl += nd.w[j] * inv * (2.0 * rdt * rdn * inv - ndt);
    if (nd.kind) sl += nd.w[j] * rdt * inv;
  }
  __shared__ double sp[256];
  sp[threadIdx.x] = dl * (1.0 / kPi) + sl * (0.5 / kPi);
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sp[threadIdx.x] += sp[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* pr = p + size_t(r) * nt;
    pr[t] = (acc ? pr[t] : 0.0) + sp[0];
  }
}

// Boundary data of point forces: one thread per node, one right-hand side
// per blockIdx.y.  The sources with a nonzero force on this right-hand side
// are listed first (warp 0, in increasing order, zero tested on the bit
// pattern) in dynamic shared memory when there is room (list = 1), so that
// each node visits only those; the sum runs in the same order either way.
__global__ void k_stokeslets(NodesView nd, int ns, const double* src, int nrhs, const double* f, double* g, int list) {
  extern __shared__ int live[];
  __shared__ int nlive;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  const double* fr = f + size_t(r) * 2 * ns;
  if (list) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      int base = 0;
      for (int s0 = 0; s0 < ns; s0 += 32) {
        const int s = s0 + lane;
        const bool nz = s < ns && ((static_cast<unsigned long long>(__double_as_longlong(fr[2 * s])) |
                                    static_cast<unsigned long long>(__double_as_longlong(fr[2 * s + 1]))) << 1) != 0ull;
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (nz) live[base + __popc(m & ((1u << lane) - 1u))] = s;
        base += __popc(m);
      }
      if (lane == 0) nlive = base;
    }
    __syncthreads();
  }
  if (i >= nd.n) return;
  const int cnt = list ? nlive : ns;
  double gx = 0.0, gy = 0.0;
  for (int q = 0; q < cnt; ++q) {
    const int s = list ? live[q] : q;
    if (!list && fr[2 * s] == 0.0 && fr[2 * s + 1] == 0.0) continue;  // no force on this right-hand side
    const double rx = nd.x[i] - src[2 * s], ry = nd.y[i] - src[2 * s + 1], r2 = rx * rx + ry * ry;
    const double lg = -0.5 * log(r2);
    const double rf = (rx * fr[2 * s] + ry * fr[2 * s + 1]) / r2;
    gx += lg * fr[2 * s] + rx * rf;
    gy += lg * fr[2 * s + 1] + ry * rf;
  }
  g[size_t(r) * 2 * nd.n + 2 * i] = gx / (4.0 * kPi);
  g[size_t(r) * 2 * nd.n + 2 * i + 1] = gy / (4.0 * kPi);
}

__global__ void k_max_colnorm(const double* W, int nr, int nc, int ld, unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= nc) return;
  double s = 0.0;
  for (int i = lane; i < nr; i += 32) { double v = W[i + size_t(j) * ld]; s += v * v; }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) atomicMax(out, __double_as_longlong(sqrt(s)));  // non-negative doubles order as integers
}

__global__ void k_to_double(const unsigned long long* in, double* out) { *out = __longlong_as_double(*in); }

__global__ void k_gather_scatter(const double* in, int ldi, const int* ii, double* out, int ldo, const int* io, int n) {
  const int r = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int a = ii ? ii[i] : i, b = io ? io[i] : i;
    out[b + size_t(r) * ldo] = in[a + size_t(r) * ldi];
  }
}

// y = A x for A = -1/2 I + D + N on one node set, evaluated on the fly
// (exact refined operator).  One thread per target point, source points
// staged through shared memory in tiles; the rank-one N term is added from
// the flux sum_j w_j n_j . x_j computed by k_flux.
constexpr int NB_T = 128, NB_S = 128;
template <int NR>
__global__ void __launch_bounds__(NB_T) k_apply_exact(NodesView nd, const double* x, int ldx, double* y, int ldy,
                                                       const double* flux, int r0) {
  // one thread per target point, up to NR right-hand sides per pass: each
  // kernel entry is evaluated once and applied to all of them
  const int i = blockIdx.x * NB_T + threadIdx.x;
  __shared__ double sx[NB_S], sy[NB_S], snx[NB_S], sny[NB_S], sw[NB_S], st[NB_S][2 * NR];
  const bool act = i < nd.n;
  const double xi = act ? nd.x[i] : 0.0, yi = act ? nd.y[i] : 0.0;
  double ux[NR], uy[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { ux[r] = 0.0; uy[r] = 0.0; }
  for (int j0 = 0; j0 < nd.n; j0 += NB_S) {
    const int nj = min(NB_S, nd.n - j0);
    __syncthreads();
    for (int q = threadIdx.x; q < nj; q += NB_T) {
      const int j = j0 + q;
      sx[q] = nd.x[j]; sy[q] = nd.y[j]; snx[q] = nd.nx[j]; sny[q] = nd.ny[j]; sw[q] = nd.w[j];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        st[q][2 * r] = x[size_t(r0 + r) * ldx + 2 * j];
        st[q][2 * r + 1] = x[size_t(r0 + r) * ldx + 2 * j + 1];
      }
    }
    __syncthreads();
    if (act) {
      for (int q = 0; q < nj; ++q) {
        if (j0 + q == i) continue;
        const double rx = xi - sx[q], ry = yi - sy[q], r2 = rx * rx + ry * ry;
        const double fac = sw[q] * (rx * snx[q] + ry * sny[q]) / (kPi * r2 * r2);
        const double fx = fac * rx, fy = fac * ry;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const double rt = rx * st[q][2 * r] + ry * st[q][2 * r + 1];
          ux[r] = fma(fx, rt, ux[r]);
          uy[r] = fma(fy, rt, uy[r]);
        }
      }
    }
  }
  if (!act) return;
  const double nxi = nd.nx[i], nyi = nd.ny[i], txi = -nyi, tyi = nxi;
  const double dkw = -nd.kappa[i] * nd.w[i] * (0.5 / kPi);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const double* xr = x + size_t(r0 + r) * ldx;
    const double taux = xr[2 * i], tauy = xr[2 * i + 1];
    const double dk = dkw * (txi * taux + tyi * tauy);
    const double fl = flux[r0 + r];
    y[size_t(r0 + r) * ldy + 2 * i] = ux[r] + dk * txi + nxi * fl - 0.5 * taux;
    y[size_t(r0 + r) * ldy + 2 * i + 1] = uy[r] + dk * tyi + nyi * fl - 0.5 * tauy;
  }
}

__global__ void k_flux(NodesView nd, const double* x, int ldx, double* flux) {
  const int r = blockIdx.x;
  const double* xr = x + size_t(r) * ldx;
  double s = 0.0;
  for (int j = threadIdx.x; j < nd.n; j += blockDim.x) s += nd.w[j] * (nd.nx[j] * xr[2 * j] + nd.ny[j] * xr[2 * j + 1]);
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) flux[r] = red[0];
}

// y[T rows] (+)= A(T, S) x for two disjoint node sets, every 2 x 2 block
// evaluated on the fly (App. B: the hole columns seen on the wall, the wall
// columns seen on the holes).  One CTA per (target point, right-hand side),
// sources split over its threads (a few hundred hole targets against tens
// of thousands of wall sources still fill the GPU).
__global__ void __launch_bounds__(128) k_apply_cross(NodesView T, NodesView Sv, const double* x, int ldx, double* y,
                                                     int ldy, int acc) {
  const int i = blockIdx.x, r = blockIdx.y;
  const double* xr = x + size_t(r) * ldx;
  double ux = 0.0, uy = 0.0;
  for (int j = threadIdx.x; j < Sv.n; j += blockDim.x) {
    const Blk2 B = a_block(T, i, Sv, j, false);
    const double a = xr[2 * j], b = xr[2 * j + 1];
    ux += B.v[0][0] * a + B.v[0][1] * b;
    uy += B.v[1][0] * a + B.v[1][1] * b;
  }
  for (int off = 16; off > 0; off >>= 1) {
    ux += __shfl_down_sync(0xffffffffu, ux, off);
    uy += __shfl_down_sync(0xffffffffu, uy, off);
  }
  __shared__ double sx[4], sy[4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sx[warp] = ux; sy[warp] = uy; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double vx = sx[0] + sx[1] + sx[2] + sx[3], vy = sy[0] + sy[1] + sy[2] + sy[3];
    double* yr = y + size_t(r) * ldy;
    yr[2 * i] = (acc ? yr[2 * i] : 0.0) + vx;
    yr[2 * i + 1] = (acc ? yr[2 * i + 1] : 0.0) + vy;
  }
}

// Dense A_pp = 1/2 I + D + S on the holes (App. B; Eq. exterior_BIE), column
// major, ld = 2 N_p.  One CTA per target point i.  The double layer is
// smooth along a hole: plain panel rule with the curvature limit on the
// diagonal.  The Stokeslet is integrated against the degree-15 interpolant
// of the density on the target's own panel and two panels on either side
// (panels equal in t, at least five per hole), with the geometry exact: a 32-point
// auxiliary Gauss rule (u_f, nu_f) on the source panel, the curve evaluated
// at its nodes, the interpolant through l_j(u_f), and for the logarithm
// Legendre product integration (generalised Gaussian quadrature corrections
// in the sense of Sec. 5: exact for the density's interpolant):
//   int log|x_i - y(s)| l_j(s) |y'(s)| ds
//     ~ sum_f [Lam_f(t) + nu_f phi(u_f)] |y'(u_f)| l_j(u_f),
//   Lam_f(t) = nu_f sum_{n<32} (2n+1)/2 P_n(u_f) M_n(t),
//   phi(s) = log|x_i - y(s)| - log|t - s|  (smooth),
// with t the target's coordinate in the source panel's [-1, 1] (the panel's
// half-width h in t scales every weight); r r^T / |r|^2 takes the auxiliary
// rule alone.  Every other pair uses the plain panel rule.
constexpr int kMaxHoles = 8;
constexpr int kNearHole = 2;  // corrected panels: cyclic distance <= 2
struct HoleSet {
  int nh;
  int off[kMaxHoles + 1];
  int P[kMaxHoles];
  double geo[kMaxHoles][5];  // a, k, R, cx, cy
};

__global__ void __launch_bounds__(128) k_hole_matrix(NodesView hv, HoleSet hs, double* A, int ld) {
  constexpr int ND = 2 * kNearHole + 1;  // corrected source panels q_i - 2 .. q_i + 2
  const int i = blockIdx.x;
  int h = 0;
  while (h + 1 < hs.nh && i >= hs.off[h + 1]) ++h;
  const int P = hs.P[h], li = i - hs.off[h], qi = li >> 4, si = li & 15;
  const double hw = kPi / P;  // half-width of a panel in t
  __shared__ double Mn[ND][kAux], lam[ND][kAux], ux[ND][kAux], uy[ND][kAux], usp[ND][kAux];
  __shared__ double wl[ND][16], tab[ND][3][16];  // log weights; r r^T / r^2 (xx, xy, yy)
  const double xi = hv.x[i], yi = hv.y[i];
  if (threadIdx.x < ND) log_moments<kAux>(c_glx[si] - 2.0 * (int(threadIdx.x) - kNearHole), Mn[threadIdx.x]);
  for (int e = threadIdx.x; e < ND * kAux; e += blockDim.x) {
    const int pd = e / kAux, f = e % kAux;
    const int q = ((qi + pd - kNearHole) % P + P) % P;
    Curve c;
    c.kind = kCurveHole;
    for (int m = 0; m < 5; ++m) c.p[m] = hs.geo[h][m];
    const Pt g = curve_eval(c, (2.0 * q + 1.0 + c_ux[f]) * hw);
    ux[pd][f] = g.x;
    uy[pd][f] = g.y;
    usp[pd][f] = sqrt(g.dx * g.dx + g.dy * g.dy);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ND * kAux; e += blockDim.x) {
    const int pd = e / kAux, f = e % kAux;
    const double u = c_ux[f];
    double p0 = 1.0, p1 = u, acc = 0.5 * Mn[pd][0] + 1.5 * u * Mn[pd][1];
    for (int n = 1; n < kAux - 1; ++n) {
      const double p2 = ((2.0 * n + 1.0) * u * p1 - n * p0) / (n + 1.0);
      p0 = p1;
      p1 = p2;
      acc += (n + 1.5) * p2 * Mn[pd][n + 1];
    }
    lam[pd][f] = c_uw[f] * acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ND * 16; e += blockDim.x) {
    const int pd = e >> 4, j = e & 15;
    const double t = c_glx[si] - 2.0 * (pd - kNearHole);
    double sl = 0.0, sxx = 0.0, sxy = 0.0, syy = 0.0;
    for (int f = 0; f < kAux; ++f) {
      const double rx = xi - ux[pd][f], ry = yi - uy[pd][f], r2 = rx * rx + ry * ry;
      const double g = usp[pd][f] * c_lag[f][j];
      const double phi = 0.5 * log(r2) - log(fabs(t - c_ux[f]));
      sl += (lam[pd][f] + c_uw[f] * phi) * g;
      const double wg = c_uw[f] * g / r2;
      sxx += wg * rx * rx;
      sxy += wg * rx * ry;
      syy += wg * ry * ry;
    }
    wl[pd][j] = hw * sl;
    tab[pd][0][j] = hw * sxx;
    tab[pd][1][j] = hw * sxy;
    tab[pd][2][j] = hw * syy;
  }
  __syncthreads();
  const double c4 = 0.25 / kPi;
  for (int j = threadIdx.x; j < hv.n; j += blockDim.x) {
    const double wj = hv.w[j];
    const int lj = j - hs.off[h];
    int d = kNearHole + 1;  // not corrected
    if (lj >= 0 && lj < 16 * P) {
      d = (lj >> 4) - qi;
      if (d > P / 2) d -= P;
      if (d < -P / 2) d += P;
    }
    double b[2][2];
    // double layer (plain rule; curvature limit at the target itself)
    if (j == i) {
      const double t[2] = {-hv.ny[i], hv.nx[i]};
      const double kap = -hv.kappa[i] * wj * (0.5 / kPi);
      for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) b[a][c] = kap * t[a] * t[c] + (a == c ? 0.5 : 0.0);
    } else {
      const double rx = xi - hv.x[j], ry = yi - hv.y[j], inv = 1.0 / (rx * rx + ry * ry);
      const double r[2] = {rx, ry};
      const double fac = wj * (rx * hv.nx[j] + ry * hv.ny[j]) * inv * inv * (1.0 / kPi);
      for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) b[a][c] = fac * r[a] * r[c];
    }
    // single layer
    if (d >= -kNearHole && d <= kNearHole) {
      const int pd = d + kNearHole, sj = lj & 15;
      const double txy[2][2] = {{tab[pd][0][sj], tab[pd][1][sj]}, {tab[pd][1][sj], tab[pd][2][sj]}};
      for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) b[a][c] += c4 * (txy[a][c] - (a == c ? wl[pd][sj] : 0.0));
    } else {
      const double rx = xi - hv.x[j], ry = yi - hv.y[j], r2 = rx * rx + ry * ry, inv = 1.0 / r2;
      const double r[2] = {rx, ry};
      const double lg = 0.5 * log(r2);
      for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) b[a][c] += c4 * wj * (r[a] * r[c] * inv - (a == c ? lg : 0.0));
    }
    for (int a = 0; a < 2; ++a)
      for (int c = 0; c < 2; ++c) A[(2 * size_t(i) + a) + (2 * size_t(j) + c) * ld] = b[a][c];
  }
}

int grid1(long long n) { return int(std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096))); }

bool g_gl_ready = false;

void ensure_gl() {
  if (g_gl_ready) return;
  double x[16], w[16];
  gauss_legendre16(x, w);
  RW_CUDA(cudaMemcpyToSymbol(c_glx, x, sizeof(x)));
  RW_CUDA(cudaMemcpyToSymbol(c_glw, w, sizeof(w)));
  double ux[kAux], uw[kAux], lag[kAux][16];
  gauss_legendre_n(kAux, ux, uw);
  // barycentric weights of the 16 nodes, then the Lagrange basis at u_f
  double bw[16];
  for (int j = 0; j < 16; ++j) {
    double pr = 1.0;
    for (int m = 0; m < 16; ++m)
      if (m != j) pr *= x[j] - x[m];
    bw[j] = 1.0 / pr;
  }
  for (int f = 0; f < kAux; ++f) {
    double den = 0.0;
    for (int j = 0; j < 16; ++j) den += bw[j] / (ux[f] - x[j]);
    for (int j = 0; j < 16; ++j) lag[f][j] = bw[j] / (ux[f] - x[j]) / den;
  }
  RW_CUDA(cudaMemcpyToSymbol(c_ux, ux, sizeof(ux)));
  RW_CUDA(cudaMemcpyToSymbol(c_uw, uw, sizeof(uw)));
  RW_CUDA(cudaMemcpyToSymbol(c_lag, lag, sizeof(lag)));
  double pn[kAux][kAux];
  for (int f = 0; f < kAux; ++f) {
    double p0 = 1.0, p1 = ux[f];
    pn[f][0] = 0.5;
    pn[f][1] = 1.5 * p1;
    for (int n = 1; n < kAux - 1; ++n) {
      const double p2 = ((2.0 * n + 1.0) * ux[f] * p1 - n * p0) / (n + 1.0);
      p0 = p1;
      p1 = p2;
      pn[f][n + 1] = (n + 1.5) * p2;
    }
  }
  RW_CUDA(cudaMemcpyToSymbol(c_pn, pn, sizeof(pn)));
  g_gl_ready = true;
}

}  // namespace

void eval_nodes(const Curve& c, const double* ta, const double* tb, int n_int, double* out, int ld,
                cudaStream_t s) {
  if (n_int <= 0) return;
  ensure_gl();
  ProfScope prof_(KC_EVAL, s);
  k_nodes<<<ceil_div(16LL * n_int, 128), 128, 0, s>>>(c, ta, tb, n_int, out, ld);
  RW_CHECK_LAUNCH();
}

void set_exterior_panels(Nodes& nd, const Curve& c, const std::vector<double>& ta, const std::vector<double>& tb,
                         cudaStream_t s) {
  require(ta.size() == tb.size() && nd.n == 16 * int(ta.size()), "exterior nodes: 16 nodes per panel");
  double x[16], w[16];
  gauss_legendre16(x, w);
  const int n = nd.n;
  nd.ht.resize(n);
  nd.htm.resize(n);
  nd.hth.resize(n);
  std::vector<double> h(size_t(3) * n);
  for (size_t p = 0; p < ta.size(); ++p) {
    const double tm = 0.5 * (ta[p] + tb[p]), th = 0.5 * (tb[p] - ta[p]);
    require(th > 0.0, "exterior nodes: empty panel");
    for (int q = 0; q < 16; ++q) {
      const size_t i = 16 * p + q;
      nd.ht[i] = tm + th * x[q];
      nd.htm[i] = tm;
      nd.hth[i] = th;
      h[i] = nd.ht[i];
      h[n + i] = tm;
      h[2 * size_t(n) + i] = th;
    }
  }
  nd.pbuf.alloc(h.size());
  RW_CUDA(cudaMemcpyAsync(nd.pbuf.p, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  RW_CUDA(cudaStreamSynchronize(s));
  nd.kind = kNodesExterior;
  nd.curve = c;
}

std::vector<std::vector<int>> ext_panel_neighbours(const Nodes& nd) {
  require(nd.kind == kNodesExterior && int(nd.htm.size()) == nd.n, "ext_panel_neighbours: not an exterior node set");
  const int np = nd.n / 16;
  std::vector<std::vector<int>> nb(np);
  for (int a = 0; a < np; ++a)
    for (int b = a + 1; b < np; ++b)
      if (ext_panels_interact(nd.htm[16 * a], nd.hth[16 * a], nd.htm[16 * b], nd.hth[16 * b])) {
        nb[a].push_back(b);
        nb[b].push_back(a);
      }
  return nb;
}

void eval_idmat(const std::vector<IdMatProb>& probs, const NodesView& S, const NodesView& E1, bool e1_same,
                const NodesView& E2, bool e2_same, cudaStream_t s) {
  if (probs.empty()) return;
  long long mx = 0;
  for (auto& p : probs) mx = std::max(mx, (long long)p.ncol * p.m);
  if (mx == 0) return;
  int max_M = 1;
  for (auto& p : probs) {
    require(p.M >= 0 && idmat_nproxy(p) <= 1024, "eval_idmat: at most 1024 proxy points");
    require(p.ncirc <= 1 || p.circ, "eval_idmat: circle list missing");
    max_M = std::max(max_M, idmat_nproxy(p));
  }
  auto d = to_device_tmp(probs, s);
  dim3 grid(std::min(grid1(mx), 1024), int(probs.size()));
  ProfScope prof_(KC_EVAL, s);
  const bool ext = S.kind == kNodesExterior;
  for (auto& p : probs) {
    require(!ext || ((p.n1 == 0 || E1.kind == kNodesExterior) && (p.n2 == 0 || E2.kind == kNodesExterior)),
            "eval_idmat: exterior candidates need exterior near sets");
    require(!p.sl_in || (ext && p.kind == 1), "eval_idmat: sl_in is for incoming exterior problems");
  }
  if (ext) {
    ensure_gl();
    k_idmat<true><<<grid, 256, 4 * size_t(max_M) * sizeof(double), s>>>(d.p, max_M, S, E1, e1_same, E2, e2_same);
  } else {
    k_idmat<false><<<grid, 256, 4 * size_t(max_M) * sizeof(double), s>>>(d.p, max_M, S, E1, e1_same, E2, e2_same);
  }
  RW_CHECK_LAUNCH();
}

void eval_blocks(const std::vector<BlockProb>& probs, const NodesView& set0, const NodesView& set1,
                 cudaStream_t s) {
  std::vector<BlockProb> ps;
  long long mx = 0;
  for (auto& p : probs) if (p.mr > 0 && p.mc > 0) { ps.push_back(p); mx = std::max(mx, (long long)p.mr * p.mc); }
  if (ps.empty()) return;
  const bool ext = set0.kind == kNodesExterior;
  require(ext == (set1.kind == kNodesExterior), "eval_blocks: exterior and other node sets mixed");
  if (!ext) {
    auto d = to_device_tmp(ps, s);
    ProfScope prof_(KC_EVAL, s);
    k_blocks<false><<<dim3(std::min(grid1(mx), 1024), int(ps.size())), 256, 0, s>>>(d.p, set0, set1);
    RW_CHECK_LAUNCH();
    return;
  }
  ensure_gl();
  // exterior walls: contiguous problems by source panel, the rest entry pair
  // by entry pair
  std::vector<BlockProb> pan, gen;
  long long npan = 0, mg = 0;
  for (auto& p : ps) {
    if (!p.rows && !p.cols) {
      pan.push_back(p);
      npan = std::max<long long>(npan, (p.c0 + p.mc - 1) / 32 - p.c0 / 32 + 1);
    } else {
      gen.push_back(p);
      mg = std::max(mg, (long long)p.mr * p.mc);
    }
  }
  TBuf<BlockProb> dp, dg;
  if (!pan.empty()) dp = to_device_tmp(pan, s);
  if (!gen.empty()) dg = to_device_tmp(gen, s);
  ProfScope prof_(KC_EVAL, s);
  if (!pan.empty()) {
    k_blocks_ext_panels<<<dim3(int(std::min<long long>(npan, 4096)), int(pan.size())), 128, 0, s>>>(dp.p, set0, set1);
    RW_CHECK_LAUNCH();
  }
  if (!gen.empty()) {
    k_blocks_ext<<<dim3(std::min(grid1(mg), 1024), int(gen.size())), 256, 0, s>>>(dg.p, set0, set1);
    RW_CHECK_LAUNCH();
  }
}

void batched_transpose(const std::vector<TransProb>& probs, cudaStream_t s) {
  std::vector<TransProb> ps;
  long long mx = 0;
  for (auto& p : probs) if (p.m > 0 && p.n > 0) { ps.push_back(p); mx = std::max(mx, (long long)p.m * p.n); }
  if (ps.empty()) return;
  auto d = to_device_tmp(ps, s);
  dim3 grid(std::min(grid1(mx), 1024), int(ps.size()));
  ProfScope prof_(KC_OTHER, s);
  k_transpose<<<grid, 256, 0, s>>>(d.p);
  RW_CHECK_LAUNCH();
}

void batched_copy(const std::vector<CopyProb>& probs, cudaStream_t s) {
  std::vector<CopyProb> ps;
  long long mx = 0;
  for (auto& p : probs) if (p.m > 0 && p.n > 0) { ps.push_back(p); mx = std::max(mx, (long long)p.m * p.n); }
  if (ps.empty()) return;
  auto d = to_device_tmp(ps, s);
  dim3 grid(std::min(grid1(mx), 1024), int(ps.size()));
  ProfScope prof_(KC_OTHER, s);
  k_copy<<<grid, 256, 0, s>>>(d.p);
  RW_CHECK_LAUNCH();
}

namespace {
int sm_count_dev() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 152;
    }
    return v;
  }();
  return n;
}
}  // namespace

void eval_velocity(const NodesView& nodes, const double* tau, int nrhs, int nt, const double* targets, double* u,
                   cudaStream_t s, int ldt, bool accumulate) {
  if (nt <= 0 || nrhs <= 0) return;
  if (nodes.n <= 0) {
    if (!accumulate) fill_zero(u, size_t(2) * nt * nrhs, s);
    return;
  }
  ProfScope prof_(KC_EVAL, s);
  // enough CTAs for the SMs: the sources are cut into chunks (at least 2048
  // each) when targets x right-hand-side groups alone are few
  const int groups = ceil_div(nrhs, kVelRhs);
  const long long ctas = (long long)nt * groups;
  const int nchunk = int(std::max(1LL, std::min<long long>(ceil_div(4LL * sm_count_dev(), ctas), nodes.n / 2048)));
  const int ld = ldt > 0 ? ldt : 2 * nodes.n;
  if (nchunk == 1) {
    k_velocity<<<dim3(nt, groups, 1), 256, 0, s>>>(nodes, tau, ld, nt, nrhs, targets, u, accumulate, nullptr);
    RW_CHECK_LAUNCH();
    return;
  }
  const size_t n = size_t(2) * nt * nrhs;
  TBuf<double> part(n * nchunk, s);
  k_velocity<<<dim3(nt, groups, nchunk), 256, 0, s>>>(nodes, tau, ld, nt, nrhs, targets, u, accumulate, part.p);
  RW_CHECK_LAUNCH();
  k_velocity_sum<<<int(std::min<size_t>((n + 255) / 256, 1024)), 256, 0, s>>>(part.p, nchunk, n, u, accumulate);
  RW_CHECK_LAUNCH();
}

void eval_pressure(const NodesView& nodes, const double* tau, int nrhs, int nt, const double* targets, double* p,
                   cudaStream_t s, int ldt, bool accumulate) {
  if (nt <= 0 || nrhs <= 0) return;
  if (nodes.n <= 0) {
    if (!accumulate) fill_zero(p, size_t(nt) * nrhs, s);
    return;
  }
  ProfScope prof_(KC_EVAL, s);
  k_pressure<<<dim3(nt, nrhs), 256, 0, s>>>(nodes, tau, ldt > 0 ? ldt : 2 * nodes.n, nt, targets, p, accumulate);
  RW_CHECK_LAUNCH();
}

void apply_cross(const NodesView& T, const NodesView& Sv, const double* x, int ldx, double* y, int ldy, int nrhs,
                 bool accumulate, cudaStream_t s) {
  if (T.n <= 0 || nrhs <= 0) return;
  require(T.kind != Sv.kind, "apply_cross: the node sets must be a wall and holes");
  ProfScope prof_(KC_EVAL, s);
  require(nrhs <= 65535, "apply_cross: at most 65535 right-hand sides per call");
  k_apply_cross<<<dim3(T.n, nrhs), 128, 0, s>>>(T, Sv, x, ldx, y, ldy, accumulate);
  RW_CHECK_LAUNCH();
}

void eval_hole_matrix(const NodesView& holes, const std::vector<int>& panels, const std::vector<double>& geo,
                      double* A, cudaStream_t s) {
  require(!panels.empty() && int(panels.size()) <= kMaxHoles, "hole matrix: 1 to 8 holes");
  require(geo.size() == 5 * panels.size(), "hole matrix: five shape parameters per hole");
  require(holes.kind == 1, "hole matrix: node set is not a hole set");
  ensure_gl();
  HoleSet hs{};
  hs.nh = int(panels.size());
  int off = 0;
  for (int h = 0; h < hs.nh; ++h) {
    require(panels[h] >= 2 * kNearHole + 1, "hole matrix: at least five panels per hole");
    hs.off[h] = off;
    hs.P[h] = panels[h];
    for (int e = 0; e < 5; ++e) hs.geo[h][e] = geo[5 * h + e];
    off += 16 * panels[h];
  }
  hs.off[hs.nh] = off;
  require(off == holes.n, "hole matrix: panel counts do not match the nodes");
  ProfScope prof_(KC_EVAL, s);
  k_hole_matrix<<<holes.n, 128, 0, s>>>(holes, hs, A, 2 * holes.n);
  RW_CHECK_LAUNCH();
}

void eval_stokeslets(const NodesView& nodes, int ns, const double* src, int nrhs, const double* f, double* g,
                     cudaStream_t s) {
  if (nodes.n <= 0 || nrhs <= 0) return;
  ProfScope prof_(KC_EVAL, s);
  const int list = ns <= 8192 ? 1 : 0;  // the list of live sources fits shared memory
  k_stokeslets<<<dim3(ceil_div(nodes.n, 128), nrhs), 128, list ? size_t(ns) * sizeof(int) : 0, s>>>(nodes, ns, src, nrhs,
                                                                                                   f, g, list);
  RW_CHECK_LAUNCH();
}

void apply_exact(const NodesView& nodes, const double* x, double* y, int nrhs, cudaStream_t s, int ldx, int ldy) {
  if (nodes.n <= 0 || nrhs <= 0) return;
  if (ldx <= 0) ldx = 2 * nodes.n;
  if (ldy <= 0) ldy = 2 * nodes.n;
  TBuf<double> flux(nrhs, s);
  ProfScope prof_(KC_EVAL, s);
  k_flux<<<nrhs, 256, 0, s>>>(nodes, x, ldx, flux.p);
  RW_CHECK_LAUNCH();
  for (int r0 = 0; r0 < nrhs; r0 += 4) {
    const int nr = std::min(4, nrhs - r0);
    const dim3 grid(ceil_div(nodes.n, NB_T));
    switch (nr) {
      case 1: k_apply_exact<1><<<grid, NB_T, 0, s>>>(nodes, x, ldx, y, ldy, flux.p, r0); break;
      case 2: k_apply_exact<2><<<grid, NB_T, 0, s>>>(nodes, x, ldx, y, ldy, flux.p, r0); break;
      case 3: k_apply_exact<3><<<grid, NB_T, 0, s>>>(nodes, x, ldx, y, ldy, flux.p, r0); break;
      default: k_apply_exact<4><<<grid, NB_T, 0, s>>>(nodes, x, ldx, y, ldy, flux.p, r0); break;
    }
    RW_CHECK_LAUNCH();
  }
}

void max_colnorm(const double* W, int nr, int nc, int ld, double* out, cudaStream_t s) {
  TBuf<unsigned long long> tmp(1, s);
  RW_CUDA(cudaMemsetAsync(tmp.p, 0, sizeof(unsigned long long), s));
  if (nc > 0) {
    k_max_colnorm<<<ceil_div(32LL * nc, 256), 256, 0, s>>>(W, nr, nc, ld, tmp.p);
    RW_CHECK_LAUNCH();
  }
  k_to_double<<<1, 1, 0, s>>>(tmp.p, out);
  RW_CHECK_LAUNCH();
}

void gather_scatter(const double* in, int ldi, const int* idx_in, double* out, int ldo, const int* idx_out, int n,
                    int nrhs, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return;
  ProfScope prof_(KC_OTHER, s);
  k_gather_scatter<<<dim3(std::min(ceil_div(n, 256), 1024), nrhs), 256, 0, s>>>(in, ldi, idx_in, out, ldo, idx_out, n);
  RW_CHECK_LAUNCH();
}

}  // namespace rw
