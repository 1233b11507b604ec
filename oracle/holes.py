"""Channel (or any wall) with added holes: App. B, with the combined-field
exterior BIE of Sec. 2 (Eq. exterior_BIE) on the holes.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Geometry.  Hole i is the closed curve
    x(t) = c_i + R_i (1 + a_i cos(k_i t)) (cos t, sin t),  t in [0, 2 pi),
counter-clockwise, cut into P_i panels equal in t with 16 Gauss-Legendre
nodes each (the paper's holes are circles, a_i = 0, with 10 panels, Sec. 5.2).
The normal n = (y', -x') / |x'| points out of the hole, into the fluid.

System (App. B, Eq. simple_ext; readings where the paper is silent):
* wall rows, wall columns:  A_kk = -1/2 I + D + N, the wall's own operator
  (Sec. 2, Remark 2.1), N over the wall points only;
* hole rows, hole columns:  A_pp = 1/2 I + D + S, the combined field of
  Eq. exterior_BIE with the hole's outward normal;
* wall rows, hole columns:  A_kp = w_j (D + S)(x_i, y_j);
* hole rows, wall columns:  A_pk = w_j D(x_i, y_j) (no N term).
The velocity in the fluid is the double layer of the wall density plus the
combined field of the hole density (Sec. 5.2: double layer on the channel,
combined field on the holes).

Quadrature.  The double layer is smooth on a smooth curve: plain Nystrom with
the curvature limit on the diagonal, as for the wall.  The Stokeslet kernel
S(x, y) = 1/(4 pi) (-log|r| I + r r^T / |r|^2) has a logarithmic singularity:
for a target on a hole and each source panel of the same hole within two
panels of it, the oracle integrates the exact kernel against the panel's
degree-15 interpolant of the density with a composite 16-point Gauss rule
graded geometrically toward the target (36 halvings on each side; the two
innermost intervals, 2^-36 of the panel, integrated in closed form with the
density frozen), a brute-force rule whose error is far below FP64 rounding.
Every other pair uses the plain panel rule.

Parity: pinned by tests/test_oracle_holes.py -- Fourier closed forms of the
logarithmic potential on a circle, the single layer of a constant density on a
circle, the closed-form Stokeslet field in the fluid for data made by
Stokeslets outside the wall and inside the holes (with spectral decay), and
planted sign and quadrature mistakes that the closed form rejects.
"""
from functools import lru_cache

import numpy as np

from .quadrature import gauss_legendre, NQ
from .curves import evaluate
from . import stokes as S

GRADE_LEVELS = 36      # halvings toward the singular point on each side
NEAR_PANELS = 2        # source panels within this cyclic distance are graded


def _hole_curve(h, t):
    g = evaluate("star", t, a=h.get("a", 0.0), k=h.get("k", 1), scale=h["R"])
    g["x"] = g["x"] + h["cx"]
    g["y"] = g["y"] + h["cy"]
    return g


def hole_nodes(holes):
    """Nodes of all holes, hole by hole, panel by panel.

    holes: list of dicts with cx, cy, R, a, k, P.  Returns the node dict of
    the wall format (x, y, nx, ny, w, kappa) plus t (parameter), hole and
    panel (indices) per node."""
    xi, om = gauss_legendre(NQ)
    parts = []
    for hi, h in enumerate(holes):
        P = int(h["P"])
        step = 2.0 * np.pi / P
        mid = (np.arange(P) + 0.5) * step
        t = (mid[:, None] + 0.5 * step * xi[None, :]).ravel()
        g = _hole_curve(h, t)
        speed = np.hypot(g["dx"], g["dy"])
        parts.append(dict(
            x=g["x"], y=g["y"], nx=g["dy"] / speed, ny=-g["dx"] / speed,
            w=(0.5 * step * om[None, :] * np.ones((P, 1))).ravel() * speed,
            kappa=(g["dx"] * g["ddy"] - g["dy"] * g["ddx"]) / speed ** 3,
            t=t, hole=np.full(t.size, hi), panel=np.repeat(np.arange(P), NQ)))
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def _bary_weights(xs):
    """Barycentric weights of Lagrange interpolation on the nodes xs."""
    d = xs[:, None] - xs[None, :]
    np.fill_diagonal(d, 1.0)
    return 1.0 / d.prod(axis=1)


def _lagrange(xs, bw, s):
    """Values of the Lagrange basis of the nodes xs at the points s: (len(s), len(xs))."""
    d = s[:, None] - xs[None, :]
    hit = d == 0.0
    d[hit] = 1.0
    terms = bw[None, :] / d
    out = terms / terms.sum(axis=1, keepdims=True)
    rows = np.where(hit.any(axis=1))[0]
    for r in rows:
        out[r] = hit[r].astype(np.float64)
    return out


@lru_cache(maxsize=None)
def _gl():
    return gauss_legendre(NQ)


@lru_cache(maxsize=256)
def _graded_rule(sstar, singular, levels):
    """Composite Gauss rule on [-1, 1] graded toward sstar in [-1, 1].

    Returns points, weights (local panel coordinate) and the lengths of the
    innermost intervals [sstar - e, sstar] and [sstar, sstar + e] when the
    kernel is singular at sstar (those two are integrated in closed form by
    the caller); otherwise the innermost intervals take the Gauss rule too.
    The result depends on sstar only (cached; callers must not modify it)."""
    xi, om = _gl()
    pts, wts, ends = [], [], []
    for side, L in ((-1.0, sstar + 1.0), (1.0, 1.0 - sstar)):
        if L <= 0.0:
            continue
        # intervals at distances [L 2^-(m+1), L 2^-m] from sstar, then the last one
        edges = [L * 0.5 ** m for m in range(levels + 1)]
        if not singular:
            edges.append(0.0)
        for m in range(len(edges) - 1):
            a, b = sstar + side * edges[m + 1], sstar + side * edges[m]
            lo, hi = min(a, b), max(a, b)
            pts.append(0.5 * (lo + hi) + 0.5 * (hi - lo) * xi)
            wts.append(0.5 * (hi - lo) * om)
        if singular:
            ends.append(edges[-1])
    s = np.concatenate(pts)
    return s, np.concatenate(wts), tuple(ends), _lagrange(xi, _bary_weights(xi), s)


def _near_single_layer(hn, holes, i, hole, panel):
    """Graded-rule integrals for target node i against the 16 nodes of one
    source panel: log part Lg (16,) = int log|x_i - y| l_j |y'| dt and the
    tensor part T (2, 2, 16) = int r_a r_b / |r|^2 l_j |y'| dt."""
    h = holes[hole]
    P = int(h["P"])
    step = 2.0 * np.pi / P
    mid = (panel + 0.5) * step
    xi, _ = _gl()
    bw = _bary_weights(xi)
    # target parameter, shifted by 2 pi to lie nearest the panel
    tau = hn["t"][i]
    tau = mid + np.remainder(tau - mid + np.pi, 2.0 * np.pi) - np.pi
    loc = (tau - mid) / (0.5 * step)
    singular = -1.0 < loc < 1.0
    sstar = float(np.clip(loc, -1.0, 1.0))
    s, ws, ends, lag = _graded_rule(sstar, singular, GRADE_LEVELS)   # lag: (nf, 16)
    g = _hole_curve(h, mid + 0.5 * step * s)
    speed = np.hypot(g["dx"], g["dy"])
    rx = hn["x"][i] - g["x"]
    ry = hn["y"][i] - g["y"]
    r2 = rx * rx + ry * ry
    base = ws * 0.5 * step * speed                      # dt = (step / 2) ds
    Lg = (base * 0.5 * np.log(r2)) @ lag
    rr = (rx, ry)
    T = np.empty((2, 2, NQ))
    for a in range(2):
        for b in range(2):
            T[a, b] = (base * rr[a] * rr[b] / r2) @ lag
    if ends:
        # innermost intervals of length e on each side of the target: the
        # density and the speed are constant to O(e), |r| = C u with
        # C = (step / 2) |x'|, so int_0^e log(C u) du = e (log(C e) - 1) and
        # r r^T / |r|^2 is the tangent's outer product
        g0 = _hole_curve(h, np.array([tau]))
        sp0 = float(np.hypot(g0["dx"], g0["dy"])[0])
        C = 0.5 * step * sp0
        l0 = _lagrange(xi, bw, np.array([sstar]))[0]
        tx, ty = float(g0["dx"][0]) / sp0, float(g0["dy"][0]) / sp0
        tt = ((tx * tx, tx * ty), (ty * tx, ty * ty))
        for e in ends:
            Lg = Lg + C * e * (np.log(C * e) - 1.0) * l0
            for a in range(2):
                for b in range(2):
                    T[a, b] = T[a, b] + C * e * tt[a][b] * l0
    return Lg, T


def _near_pairs(hn, holes):
    """(target i, hole, source panel) triples that take the graded rule."""
    out = []
    for i in range(hn["x"].size):
        hole, pi = int(hn["hole"][i]), int(hn["panel"][i])
        P = int(holes[hole]["P"])
        seen = set()
        for d in range(-NEAR_PANELS, NEAR_PANELS + 1):
            q = (pi + d) % P
            if q not in seen:
                seen.add(q)
                out.append((i, hole, q))
    return out


def _panel_cols(hn, holes, hole, panel):
    off = sum(NQ * int(holes[j]["P"]) for j in range(hole))
    return off + NQ * panel + np.arange(NQ)


def log_matrix(hn, holes):
    """Scalar matrix Lw (N x N) with (Lw f)_i ~ int log|x_i - y| f(y) ds_y over
    all holes: plain panel rule, graded rule on the near panels."""
    rx = hn["x"][:, None] - hn["x"][None, :]
    ry = hn["y"][:, None] - hn["y"][None, :]
    r2 = rx * rx + ry * ry
    np.fill_diagonal(r2, 1.0)
    Lw = 0.5 * np.log(r2) * hn["w"][None, :]
    for i, hole, q in _near_pairs(hn, holes):
        cols = _panel_cols(hn, holes, hole, q)
        Lw[i, cols] = _near_single_layer(hn, holes, i, hole, q)[0]
    return Lw


def single_layer_matrix(hn, holes):
    """Stokes single layer on the holes (2N x 2N, interleaved): entries
    w_j S(x_i, y_j) with the graded rule on the near panels."""
    N = hn["x"].size
    rx = hn["x"][:, None] - hn["x"][None, :]
    ry = hn["y"][:, None] - hn["y"][None, :]
    r2 = rx * rx + ry * ry
    np.fill_diagonal(r2, 1.0)
    w = hn["w"][None, :]
    lg = 0.5 * np.log(r2)
    rr = (rx, ry)
    c = 1.0 / (4.0 * np.pi)
    M = np.empty((2 * N, 2 * N))
    for a in range(2):
        for b in range(2):
            M[a::2, b::2] = c * w * ((-lg if a == b else 0.0) + rr[a] * rr[b] / r2)
    for i, hole, q in _near_pairs(hn, holes):
        cols = _panel_cols(hn, holes, hole, q)
        Lg, T = _near_single_layer(hn, holes, i, hole, q)
        for a in range(2):
            for b in range(2):
                M[2 * i + a, 2 * cols + b] = c * ((-Lg if a == b else 0.0) + T[a, b])
    return M


def double_layer_matrix(hn):
    """Double layer on the holes (2N x 2N): w_j D(x_i, y_j), the curvature
    limit -(kappa_i w_i / 2 pi) t_i t_i^T on the diagonal, no N term."""
    x, y, nx, ny, w, kap = hn["x"], hn["y"], hn["nx"], hn["ny"], hn["w"], hn["kappa"]
    N = x.size
    rx = x[:, None] - x[None, :]
    ry = y[:, None] - y[None, :]
    r2 = rx * rx + ry * ry
    np.fill_diagonal(r2, 1.0)
    fac = w[None, :] * (rx * nx[None, :] + ry * ny[None, :]) / (np.pi * r2 * r2)
    rr = (rx, ry)
    tt = (-ny, nx)
    d = -kap * w / (2.0 * np.pi)
    M = np.empty((2 * N, 2 * N))
    ii = np.arange(N)
    for a in range(2):
        for b in range(2):
            blk = fac * rr[a] * rr[b]
            blk[ii, ii] = d * tt[a] * tt[b]
            M[a::2, b::2] = blk
    return M


def hole_matrix(hn, holes, jump=0.5):
    """A_pp = jump I + D + S on the holes (jump = +1/2 by Eq. exterior_BIE)."""
    return jump * np.eye(2 * hn["x"].size) + double_layer_matrix(hn) + single_layer_matrix(hn, holes)


def cross_double(rows, cols):
    """w_j D(x_i, y_j) for disjoint node sets (no N term): (2 nr x 2 nc)."""
    rx = rows["x"][:, None] - cols["x"][None, :]
    ry = rows["y"][:, None] - cols["y"][None, :]
    r2 = rx * rx + ry * ry
    fac = cols["w"][None, :] * (rx * cols["nx"][None, :] + ry * cols["ny"][None, :]) / (np.pi * r2 * r2)
    rr = (rx, ry)
    M = np.empty((2 * rows["x"].size, 2 * cols["x"].size))
    for a in range(2):
        for b in range(2):
            M[a::2, b::2] = fac * rr[a] * rr[b]
    return M


def cross_single(rows, cols):
    """w_j S(x_i, y_j) for disjoint node sets: (2 nr x 2 nc)."""
    rx = rows["x"][:, None] - cols["x"][None, :]
    ry = rows["y"][:, None] - cols["y"][None, :]
    r2 = rx * rx + ry * ry
    w = cols["w"][None, :]
    lg = 0.5 * np.log(r2)
    rr = (rx, ry)
    M = np.empty((2 * rows["x"].size, 2 * cols["x"].size))
    for a in range(2):
        for b in range(2):
            M[a::2, b::2] = w * ((-lg if a == b else 0.0) + rr[a] * rr[b] / r2) / (4.0 * np.pi)
    return M


def system(wall, hn, holes, jump=0.5):
    """Dense A_nn of App. B (Eq. simple_ext): unknowns ordered wall then holes."""
    Akk = S.matrix(wall)
    Akp = cross_double(wall, hn) + cross_single(wall, hn)
    Apk = cross_double(hn, wall)
    App = hole_matrix(hn, holes, jump)
    return np.block([[Akk, Akp], [Apk, App]])


def boundary_data(wall, hn, sx, sy, f):
    """Dirichlet data at the wall and hole nodes (wall first)."""
    return np.concatenate([S.boundary_data(wall, sx, sy, f), S.boundary_data(hn, sx, sy, f)])


def solve(wall, hn, holes, g):
    """Dense LU solve of the App. B system."""
    return np.linalg.solve(system(wall, hn, holes), g)


def velocity(wall, hn, tau, tx, ty):
    """Fluid velocity: wall double layer plus hole combined field.  The hole
    single layer is the Stokeslet field of the point forces w_j tau_j at the
    hole nodes (its plain panel rule, valid away from the holes)."""
    tau = np.asarray(tau, dtype=np.float64)
    nk = 2 * wall["x"].size
    tk, tp = tau[:nk], tau[nk:]
    u = S.velocity(wall, tk, tx, ty) + S.velocity(hn, tp, tx, ty)
    if tp.ndim == 1:
        f = np.stack([hn["w"] * tp[0::2], hn["w"] * tp[1::2]], axis=1)
    else:
        f = np.stack([hn["w"][:, None] * tp[0::2], hn["w"][:, None] * tp[1::2]], axis=1)
    return u + S.stokeslet_velocity(tx, ty, hn["x"], hn["y"], f)


def pressure(wall, hn, tau, tx, ty):
    """Fluid pressure of the same representation: double-layer pressure of
    both densities plus the Stokeslet pressure of the hole point forces."""
    tau = np.asarray(tau, dtype=np.float64)
    nk = 2 * wall["x"].size
    tk, tp = tau[:nk], tau[nk:]
    p = S.pressure(wall, tk, tx, ty) + S.pressure(hn, tp, tx, ty)
    if tp.ndim == 1:
        f = np.stack([hn["w"] * tp[0::2], hn["w"] * tp[1::2]], axis=1)
    else:
        f = np.stack([hn["w"][:, None] * tp[0::2], hn["w"][:, None] * tp[1::2]], axis=1)
    return p + S.stokeslet_pressure(tx, ty, hn["x"], hn["y"], f)


def apply_rows(wall, hn, holes, tau, rows, App=None):
    """(A_nn tau)[rows] without forming A_kk: wall rows one at a time from the
    wall operator's definition plus the holes' combined field; hole rows from
    the wall double layer plus the dense A_pp (passed in, or formed here)."""
    tau = np.asarray(tau, dtype=np.float64)
    squeeze = tau.ndim == 1
    if squeeze:
        tau = tau[:, None]
    nk = 2 * wall["x"].size
    tk, tp = tau[:nk], tau[nk:]
    rows = np.asarray(rows)
    out = np.empty((rows.size, tau.shape[1]))
    wr = rows < nk
    if wr.any():
        r = rows[wr]
        pts = np.unique(r // 2)
        sub = {k: wall[k][pts] for k in ("x", "y", "nx", "ny", "w", "kappa")}
        cross = (cross_double(sub, hn) + cross_single(sub, hn)) @ tp
        pos = {int(p): q for q, p in enumerate(pts)}
        own = S.apply_rows(wall, tk, r)
        out[wr] = own + np.stack([cross[2 * pos[int(d) // 2] + (int(d) & 1)] for d in r])
    hr = ~wr
    if hr.any():
        if App is None:
            App = hole_matrix(hn, holes)
        r = rows[hr] - nk
        pts = np.unique(r // 2)
        sub = {k: hn[k][pts] for k in ("x", "y", "nx", "ny", "w", "kappa")}
        pos = {int(p): q for q, p in enumerate(pts)}
        cross = cross_double(sub, wall) @ tk
        out[hr] = np.stack([cross[2 * pos[int(d) // 2] + (int(d) & 1)] for d in r]) + App[r] @ tp
    return out[:, 0] if squeeze else out
