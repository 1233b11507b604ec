"""Exterior Stokes problem on one closed wall (Sec. 2.2, Eq. exterior_BIE), on
the reference discretisation and on a locally refined one (Sec. 3.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The fluid fills the plane outside a closed counter-clockwise curve; the normal
n = (y', -x') / |x'| points out of the curve, into the fluid.  The velocity is
the combined field u = (D + S) tau, and the density solves

    1/2 tau + (D + S) tau = g   on the curve          (Eq. exterior_BIE),

a second-kind equation whose matrix is full rank: no N term.

Discretisation.  Panels are parameter intervals [a_p, b_p] with 16
Gauss-Legendre nodes each: P equal panels for the reference wall; for a
refinement, every cut panel replaced in place by 2^L equal sub-panels (the
refined order of discretize.refine).
* D: the plain panel rule, with the curvature limit on the diagonal (smooth on
  a smooth curve), plus the jump +1/2 I.
* S = 1/(4 pi) (-log|r| I + r r^T / |r|^2): for a target x_i and a source panel
  whose parameter interval, mapped to [-1, 1], puts the target's parameter at
  |loc| < NEAR_LOC (periodic distance), the exact kernel is integrated
  against the panel's degree-15 interpolant of the density by the graded
  brute-force rule of oracle/holes.py, with the geometry exact.  Its depth
  on each side stops where the parameter's rounding would merge nodes with
  the target (_grade_levels).  Every other pair takes the plain rule.  NEAR_LOC = 5 covers two equal panels on either
  side (the holes' choice).  On a refined mesh it also covers every fine panel
  next to a coarse one, and every coarse panel next to a fine one.
* Velocity at a point of the fluid: the plain panel rule (targets away from
  the curve).

Why the closed form holds.  Take Stokeslets inside the curve with total force
F.  At infinity, their field and the combined field both behave as
1/(4 pi) (-log|x| I + x x^T / |x|^2) F' + O(1 / |x|), with no constant term.
F' = F for the Stokeslets, and F' = the density's total force
sum_j w_j tau_j for the combined field.  The 2D exterior Stokes problem has
exactly one solution of that form.  A homogeneous solution of that form
would, for a circle of radius R, have to carry the constant
(1/2 - log R) F' / (4 pi), which is nonzero unless R = e^(1/2).  So the
solved field equals the Stokeslet field, and the total forces agree.

Parity: pinned by tests/test_oracle_exterior.py.
* The closed-form Stokeslet field in the fluid, with spectral decay, on the
  reference star and on refined stars.
* The total-force identity.
* Equality with the pinned combined-field hole matrix of oracle/holes.py for
  one equal-panel curve.
* The refined node order against discretize.refine.
* Planted mistakes break the closed form: the interior jump, the plain rule
  on the log singularity, and the single layer's sign.
* The extended linear system (Sec. 3.2) built from the exterior operator
  reproduces the refined exterior solve, and the Woodbury formula with exact
  and truncated-SVD factors of Q does too (the Remark closing Sec. 3.1: the
  method applies to exterior problems unchanged).
"""
from functools import lru_cache

import numpy as np

from .quadrature import NQ
from .curves import evaluate
from .discretize import _nodes_on_intervals
from . import holes as H
from . import stokes as S

NEAR_LOC = 5.0   # graded rule where the target sits within this many source half-widths
JUMP = 0.5       # +1/2 I of Eq. exterior_BIE


def panels(n_panels, cut=(), levels=()):
    """Parameter intervals (a, b) of the reference panels, or of the refined
    discretisation in refined order: the original panels 0..P-1, each cut
    panel replaced by its 2^L equal sub-panels in increasing t."""
    h = 2.0 * np.pi / n_panels
    lev = dict(zip([int(j) for j in cut], [int(L) for L in levels]))
    a, b = [], []
    for j in range(n_panels):
        ns = 2 ** lev[j] if j in lev else 1
        for q in range(ns):
            a.append(j * h + q * (h / ns))
            b.append(j * h + (q + 1) * (h / ns))
    return np.asarray(a), np.asarray(b)


def nodes(kind, params, a, b):
    """Nodes on the panels [a_p, b_p] (16 each, in panel order), with each
    node's panel index."""
    nd = _nodes_on_intervals(kind, params, a, b)
    nd["panel"] = np.repeat(np.arange(a.size), NQ)
    nd["pa"], nd["pb"] = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return nd


def _grade_levels(L, half, tau):
    """Halvings of the graded rule on a side of length L (panel coordinate)
    toward the target.  The grading stops where the innermost interval is
    1e4 rounding units of the parameter long: closer nodes would merge with
    the target's parameter.  Then e = L 2^-levels stays below 2e-11 / half
    in the panel coordinate.  The closed-form innermost piece freezes the
    density there and errs by O(e^2 log e), far below rounding."""
    if L <= 0.0:
        return 0   # no interval on this side
    floor_t = 1e4 * np.spacing(abs(tau) + 2.0 * np.pi)
    return int(np.clip(np.floor(np.log2(L * half / floor_t)), 8, 60))


@lru_cache(maxsize=4096)
def _graded_rule(sstar, singular, lev_left, lev_right):
    """Composite Gauss rule on [-1, 1] graded toward sstar, lev_left /
    lev_right halvings on either side.  Otherwise it is the rule of
    oracle/holes.py: with a singular kernel, the two innermost intervals are
    left to the caller's closed form (their lengths returned)."""
    xi, om = H._gl()
    pts, wts, ends = [], [], []
    for side, L, lev in ((-1.0, sstar + 1.0, lev_left), (1.0, 1.0 - sstar, lev_right)):
        if L <= 0.0:
            continue
        edges = [L * 0.5 ** m for m in range(lev + 1)]
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
    return s, np.concatenate(wts), tuple(ends), H._lagrange(xi, H._bary_weights(xi), s)


def _near_single_layer(kind, params, nd, i, a, b):
    """Graded-rule integrals for target node i against the 16 nodes of the
    source panel [a, b]: log part Lg (16,) = int log|x_i - y| l_j |y'| dt and
    the tensor part T (2, 2, 16) = int r_a r_b / |r|^2 l_j |y'| dt."""
    mid, half = 0.5 * (a + b), 0.5 * (b - a)
    tau = mid + np.remainder(nd["t"][i] - mid + np.pi, 2.0 * np.pi) - np.pi
    loc = (tau - mid) / half
    singular = -1.0 < loc < 1.0
    sstar = float(np.clip(loc, -1.0, 1.0))
    s, ws, ends, lag = _graded_rule(sstar, singular, _grade_levels(sstar + 1.0, half, tau),
                                    _grade_levels(1.0 - sstar, half, tau))
    g = evaluate(kind, mid + half * s, **params)
    speed = np.hypot(g["dx"], g["dy"])
    rx = nd["x"][i] - g["x"]
    ry = nd["y"][i] - g["y"]
    r2 = rx * rx + ry * ry
    base = ws * half * speed                         # dt = half ds
    Lg = (base * 0.5 * np.log(r2)) @ lag
    rr = (rx, ry)
    T = np.empty((2, 2, NQ))
    for p in range(2):
        for q in range(2):
            T[p, q] = (base * rr[p] * rr[q] / r2) @ lag
    if ends:
        # the two innermost intervals (length e on each side of the target):
        # density and speed constant to O(e), |r| = C u with C = half |x'|
        xi, _ = H._gl()
        g0 = evaluate(kind, np.array([tau]), **params)
        sp0 = float(np.hypot(g0["dx"], g0["dy"])[0])
        C = half * sp0
        l0 = H._lagrange(xi, H._bary_weights(xi), np.array([sstar]))[0]
        tx, ty = float(g0["dx"][0]) / sp0, float(g0["dy"][0]) / sp0
        tt = ((tx * tx, tx * ty), (ty * tx, ty * ty))
        for e in ends:
            Lg = Lg + C * e * (np.log(C * e) - 1.0) * l0
            for p in range(2):
                for q in range(2):
                    T[p, q] = T[p, q] + C * e * tt[p][q] * l0
    return Lg, T


def near_panels(nd, i):
    """Source panels that take the graded rule for target node i."""
    mid = 0.5 * (nd["pa"] + nd["pb"])
    half = 0.5 * (nd["pb"] - nd["pa"])
    d = np.remainder(nd["t"][i] - mid + np.pi, 2.0 * np.pi) - np.pi
    return np.nonzero(np.abs(d / half) < NEAR_LOC)[0]


def single_layer_matrix(kind, params, nd):
    """w_j S(x_i, y_j) on the curve (2N x 2N, interleaved), the graded rule
    on the near panels."""
    N = nd["x"].size
    rx = nd["x"][:, None] - nd["x"][None, :]
    ry = nd["y"][:, None] - nd["y"][None, :]
    r2 = rx * rx + ry * ry
    np.fill_diagonal(r2, 1.0)
    w = nd["w"][None, :]
    lg = 0.5 * np.log(r2)
    rr = (rx, ry)
    c = 1.0 / (4.0 * np.pi)
    M = np.empty((2 * N, 2 * N))
    for p in range(2):
        for q in range(2):
            M[p::2, q::2] = c * w * ((-lg if p == q else 0.0) + rr[p] * rr[q] / r2)
    for i in range(N):
        for pn in near_panels(nd, i):
            cols = NQ * pn + np.arange(NQ)
            Lg, T = _near_single_layer(kind, params, nd, i, nd["pa"][pn], nd["pb"][pn])
            for p in range(2):
                for q in range(2):
                    M[2 * i + p, 2 * cols + q] = c * ((-Lg if p == q else 0.0) + T[p, q])
    return M


def matrix(kind, params, nd):
    """Dense 1/2 I + D + S on the curve's nodes (2N x 2N, interleaved)."""
    return (JUMP * np.eye(2 * nd["x"].size) + H.double_layer_matrix(nd)
            + single_layer_matrix(kind, params, nd))


def solve(kind, params, nd, g):
    """Dense LU solve of the exterior system."""
    return np.linalg.solve(matrix(kind, params, nd), g)


def velocity(nd, tau, tx, ty):
    """u = (D + S) tau at points of the fluid: the double layer plus the
    Stokeslet field of the point forces w_j tau_j at the nodes."""
    tau = np.asarray(tau, dtype=np.float64)
    u = S.velocity(nd, tau, tx, ty)
    if tau.ndim == 1:
        f = np.stack([nd["w"] * tau[0::2], nd["w"] * tau[1::2]], axis=1)
    else:
        f = np.stack([nd["w"][:, None] * tau[0::2], nd["w"][:, None] * tau[1::2]], axis=1)
    return u + S.stokeslet_velocity(tx, ty, nd["x"], nd["y"], f)


def total_force(nd, tau):
    """sum_j w_j tau_j (2,) or (2, nrhs)."""
    tau = np.asarray(tau, dtype=np.float64)
    w = nd["w"] if tau.ndim == 1 else nd["w"][:, None]
    return np.stack([(w * tau[0::2]).sum(0), (w * tau[1::2]).sum(0)])


def extended_system(kind, params, n_panels, cut, levels):
    """The extended linear system of Sec. 3.2 for an exterior wall: A_ext =
    A~ + Q in the ordering [o ; p] (original points in panel order, then the
    added points in window order), A~ = blkdiag(A_oo, A_pp) and the three
    nonzero blocks of Q (-A_kc, A_kp, A_pk), every block from this module's
    exterior operator on the panels it involves.  Returns the dict of
    dense.extended_system (A_ext, At, Q, dk, dc, dp, No, Np) together with the
    refinement's bookkeeping from discretize.refine (for dense.g_ext and
    dense.ext_to_n)."""
    from .discretize import refine, dof
    ref = refine(kind, params, n_panels, list(cut), list(levels))
    ao, bo = panels(n_panels)
    h = 2.0 * np.pi / n_panels
    ap, bp = [], []
    for j, L in zip(cut, levels):
        ns = 2 ** int(L)
        for q in range(ns):
            ap.append(j * h + q * (h / ns))
            bp.append(j * h + (q + 1) * (h / ns))
    a = np.concatenate([ao, np.asarray(ap)])
    b = np.concatenate([bo, np.asarray(bp)])
    allpts = nodes(kind, params, a, b)
    No, Np = ao.size * NQ, len(ap) * NQ
    Abig = matrix(kind, params, allpts)
    dk, dc = dof(ref["I_k"]), dof(ref["I_c"])
    dp = 2 * No + np.arange(2 * Np)
    Aext = Abig.copy()
    Aext[np.ix_(dk, dc)] = 0.0
    Aext[np.ix_(dc, dp)] = 0.0
    Aext[np.ix_(dp, dc)] = 0.0
    At = np.zeros_like(Abig)
    At[:2 * No, :2 * No] = Abig[:2 * No, :2 * No]
    At[2 * No:, 2 * No:] = Abig[2 * No:, 2 * No:]
    return dict(A_ext=Aext, At=At, Q=Aext - At, dk=dk, dc=dc, dp=dp, No=No, Np=Np, ref=ref, nodes=allpts)
