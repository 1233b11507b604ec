// Geometry and kernel-matrix evaluation: wall and refined nodes from the
// curve description, entries of A on index lists, and the proxy-augmented
// matrices whose interpolative decompositions give the HBS bases and the
// low-rank factors of Q.
#pragma once
#include <cmath>
#include "rw_common.cuh"

namespace rw {

// Gauss-Legendre nodes/weights of the 16-point rule on [-1, 1] (host table,
// Newton iteration on the Legendre recurrence).
void gauss_legendre16(double* x, double* w);
void gauss_legendre_n(int n, double* x, double* w);

// Nodes on t-intervals [ta[i], tb[i]] (16 Gauss-Legendre points each) into
// `out` (6 x 16 n_int, see Nodes).  ta/tb are device arrays.
void eval_nodes(const Curve& c, const double* ta, const double* tb, int n_int,
                double* out, int ld, cudaStream_t s);

// Exterior walls (node sets of kind kNodesExterior; Sec. 2.2).  A target at
// parameter t takes the singular rule of the single layer against a source
// panel with midpoint tm and half-width th (in t) when the periodic distance
// |t - tm| is below kExtNear th.  Beyond that, the plain 16-point rule errs by
// about (2 + sqrt 3)^-32 ~ 5e-19 relative: the logarithm's singularity lies
// outside the Bernstein ellipse of parameter 2 + sqrt 3.  Node sets of this
// kind are panel aligned: the
// nodes 16 p .. 16 p + 15 are panel p's Gauss-Legendre points in order.
constexpr double kExtNear = 2.0;
__host__ __device__ inline double ext_loc(double t, double tm, double th) {
  const double twopi = 2.0 * kPi;
  double d = t - tm;
  d -= twopi * floor((d + kPi) / twopi);
  return d / th;
}
// Whether some node of panel a takes the singular rule against panel b or
// some node of b against a (whole panels: a conservative test).
inline bool ext_panels_interact(double tma, double tha, double tmb, double thb) {
  const double d = std::fabs(ext_loc(tma, tmb, 1.0));
  return d - tha < kExtNear * thb || d - thb < kExtNear * tha;
}
// Make nd an exterior-wall node set on curve c whose panels are the
// t-intervals [ta[p], tb[p]] (nd.n = 16 x panels): kind, curve, and the
// per-node t, tm, th on the host and the device.
void set_exterior_panels(Nodes& nd, const Curve& c, const std::vector<double>& ta, const std::vector<double>& tb,
                         cudaStream_t s);
// For each panel of an exterior node set, the other panels that share a
// singular-rule pair with it (ext_panels_interact).
std::vector<std::vector<int>> ext_panel_neighbours(const Nodes& nd);

// Internal curve kind of a hole: x(t) = c + R (1 + a cos(k t)) (cos t, sin t),
// p = {a, k, R, cx, cy} (counter-clockwise; the normal points into the fluid).
constexpr int kCurveHole = 100;

// Columns of an ID matrix, written transposed: W (ncol x m) holds Y^T.
// kind 0 ("outgoing", rows of A): Y[i, :] = [A(cand_i, e1) | A(cand_i, e2) |
//   S(x_i, z_q) e_b, D(x_i, z_q) e_b for proxy points z_q | n_i]
// kind 1 ("incoming", columns of A): Y[i, :] = [A(e1, cand_i)^T |
//   A(e2, cand_i)^T | w_i D(z_q, x_i)[a', .] for proxy points | w_i n_i],
//   with sl_in also w_i S(z_q, x_i)[a', .] after the double layer's columns.
// Candidates live in node set S; e1 in E1 and e2 in E2.  Proxy points are
// z_q = c + R (cos 2 pi q / M, sin 2 pi q / M) with outward normal; with
// ncirc > 1 the proxies are the union of M points on each of the circles
// circ[3 c .. 3 c + 2] = (cx, cy, R) (device array), as for several holes.
struct IdMatProb {
  int kind;
  int m;
  const int* cand;
  int n1;
  const int* e1;
  int n2;
  const int* e2;
  double cx, cy, R;
  int M;
  int normal;
  double* W;
  int ldw;
  int ncol;
  int ncirc;
  const double* circ;
  int sl_in;  // kind 1 on exterior-wall candidates: the single layer's field
              // at the proxy points too (2 more columns per proxy point)
};
inline int idmat_nproxy(const IdMatProb& p) { return p.M * (p.ncirc > 1 ? p.ncirc : 1); }
inline int idmat_ncol(int kind, int n1, int n2, int M, int normal, int sl_in = 0) {
  return n1 + n2 + ((kind == 0 || sl_in) ? 4 * M : 2 * M) + (normal ? 1 : 0);
}
void eval_idmat(const std::vector<IdMatProb>& probs, const NodesView& S,
                const NodesView& E1, bool e1_same, const NodesView& E2,
                bool e2_same, cudaStream_t s);

// Dense blocks out (mr x mc, ld) = scale * A(rows, cols); rows index DOFs of
// node set sets[rset], cols of sets[cset] (rset == cset: same set, with the
// diagonal blocks).  rows == nullptr means rows r0 .. r0+mr-1 (same for cols).
struct BlockProb {
  int mr, mc;
  const int* rows;
  const int* cols;
  int r0, c0;
  int rset, cset;
  double scale;
  double* out;
  int ld;
};
void eval_blocks(const std::vector<BlockProb>& probs, const NodesView& set0,
                 const NodesView& set1, cudaStream_t s);

// out (n x m, ldo) = in^T (in: m x n, ldi), batched.
struct TransProb {
  const double* in;
  int m, n, ldi;
  double* out;
  int ldo;
};
void batched_transpose(const std::vector<TransProb>& probs, cudaStream_t s);

// out[r0:r0+m, c0:c0+n] (ldo) = in (m x n, ldi), batched copies of blocks.
struct CopyProb {
  const double* in;
  int m, n, ldi;
  double* out;
  int ldo;
};
void batched_copy(const std::vector<CopyProb>& probs, cudaStream_t s);

// Velocity u(x) = sum_j w_j D(x, y_j) tau_j at targets (Sec. 2.1); a hole
// set (kind 1) adds its single layer sum_j w_j S(x, y_j) tau_j (App. B).
// targets: 2 x nt; tau: 2N x nrhs (ld ldt, default 2N); u: 2nt x nrhs (ld
// 2nt), overwritten or accumulated into.
void eval_velocity(const NodesView& nodes, const double* tau, int nrhs, int nt,
                   const double* targets, double* u, cudaStream_t s, int ldt = 0, bool accumulate = false);

// Pressure of the same representation at targets (Sec. 2): p (nt x nrhs).
void eval_pressure(const NodesView& nodes, const double* tau, int nrhs, int nt, const double* targets, double* p,
                   cudaStream_t s, int ldt = 0, bool accumulate = false);

// y[T] (+)= A(T, S) x between a wall set and a hole set (either order),
// entries evaluated on the fly; x: 2 S.n x nrhs (ld ldx), y: 2 T.n x nrhs.
void apply_cross(const NodesView& T, const NodesView& S, const double* x, int ldx, double* y, int ldy, int nrhs,
                 bool accumulate, cudaStream_t s);

// Dense A_pp = 1/2 I + D + S on a hole set whose hole h has panels[h] equal
// panels in t (16 points each, in order) and shape geo[5h .. 5h+4] = (a, k,
// R, cx, cy) (kCurveHole): A is 2N x 2N column major.
void eval_hole_matrix(const NodesView& holes, const std::vector<int>& panels, const std::vector<double>& geo,
                      double* A, cudaStream_t s);

// g(x_i) = sum_s S(x_i, y_s) f_s (Eq. stokeslet, mu = 1) at every node.
// src: 2 x ns; f: 2 x ns x nrhs; g: 2N x nrhs.
void eval_stokeslets(const NodesView& nodes, int ns, const double* src,
                     int nrhs, const double* f, double* g, cudaStream_t s);

// y = A x with A = -1/2 I + D + N on a node set, every entry evaluated on
// the fly (the exact Nystrom operator of Sec. 2).  x, y: 2N x nrhs, ld 2N.
void apply_exact(const NodesView& nodes, const double* x, double* y, int nrhs, cudaStream_t s, int ldx = 0,
                 int ldy = 0);

// Row-norm maximum of a column-major W (nr x nc): max_j ||W[:, j]|| into out.
void max_colnorm(const double* W, int nr, int nc, int ld, double* out,
                 cudaStream_t s);

// Scatter/gather of interleaved DOF vectors: out[idx_out[i]] = in[idx_in[i]]
// for i < n and every right-hand side (column strides ldi/ldo).
void gather_scatter(const double* in, int ldi, const int* idx_in, double* out,
                    int ldo, const int* idx_out, int n, int nrhs,
                    cudaStream_t s);

}  // namespace rw
