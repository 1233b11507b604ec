"""The singular rule of the exterior wall's CUDA entries, restated on the CPU
and checked entry by entry against oracle/exterior.py's graded rule.

The CUDA path integrates the single layer's logarithm near each target by
Legendre product integration on a 32-point auxiliary rule (Sec. 5: quadrature
corrections exact for the density's panel interpolant).  The moments
M_n(t) = int P_n(s) log|t - s| ds come from the Legendre functions of the
second kind: the forward recurrence inside the panel, Miller's backward
recurrence outside.  The oracle integrates the same kernel against the same
interpolant by brute force on a geometrically graded composite Gauss rule.
This test writes the product rule out in numpy (a statement of the formula,
independent of both the CUDA code and the oracle).  It checks the two weight
sets against each other for the pairs the CUDA path corrects: a target on its
own panel, a coarse target next to a level-5 run of fine panels, and fine
targets next to the coarse panel.  The relative agreement is 1e-11 or better.
"""
import numpy as np

from oracle import exterior as X
from oracle.curves import evaluate

STAR = dict(a=0.3, k=5)
NA = 32


def _moments(t, nm=NA):
    """M_n(t), n < nm, from Q_n(t) (M_n = 2 (Q_{n+1} - Q_{n-1}) / (2n + 1))."""
    Q = np.zeros(nm + 1)
    if abs(t) < 1.0:
        Q[0] = 0.5 * np.log((1.0 + t) / (1.0 - t))
        Q[1] = t * Q[0] - 1.0
        for n in range(1, nm):
            Q[n + 1] = ((2 * n + 1) * t * Q[n] - n * Q[n - 1]) / (n + 1)
    else:
        rho = abs(t) + np.sqrt((abs(t) - 1.0) * (abs(t) + 1.0))
        n0 = nm + 1 + int(np.ceil(40.0 / np.log(rho)))
        q_hi, q = 0.0, 1.0
        vals = {}
        for n in range(n0, 0, -1):
            q_lo = ((2 * n + 1) * t * q - (n + 1) * q_hi) / n
            q_hi, q = q, q_lo
            vals[n - 1] = q
            if abs(q) > 1e200:
                q *= 1e-200
                q_hi *= 1e-200
                for m in vals:
                    vals[m] *= 1e-200
        for m in range(nm + 1):
            Q[m] = vals[m]
        Q *= 0.5 * np.log((t + 1.0) / (t - 1.0)) / Q[0]
    M = np.empty(nm)
    M[0] = (t + 1.0) * np.log(abs(t + 1.0)) - (t - 1.0) * np.log(abs(t - 1.0)) - 2.0
    for n in range(1, nm):
        M[n] = 2.0 * (Q[n + 1] - Q[n - 1]) / (2 * n + 1)
    return M


def _product_rule(xi, yi, loc, tm, th):
    """Weights (16,) of int log|x - y| l_q |y'| dt and (2, 2, 16) of
    int r_a r_b / |r|^2 l_q |y'| dt on the panel (tm - th, tm + th)."""
    u, w = np.polynomial.legendre.leggauss(NA)
    xg, _ = np.polynomial.legendre.leggauss(16)
    bw = np.array([1.0 / np.prod([xg[j] - xg[m] for m in range(16) if m != j]) for j in range(16)])
    terms = bw[None, :] / (u[:, None] - xg[None, :])
    lag = terms / terms.sum(axis=1, keepdims=True)                      # (NA, 16)
    P = np.polynomial.legendre.legvander(u, NA - 1)                     # P_n(u_f)
    lam = w * ((P * (np.arange(NA) + 0.5)) @ _moments(loc))
    g = evaluate("star", tm + th * u, **STAR)
    sp = np.hypot(g["dx"], g["dy"])
    rx, ry = xi - g["x"], yi - g["y"]
    r2 = rx * rx + ry * ry
    phi = 0.5 * np.log(r2 / (loc - u) ** 2)
    Lg = th * ((lam + w * phi) * sp) @ lag
    bt = w * sp / r2
    rr = (rx, ry)
    T = np.array([[th * (bt * rr[a] * rr[b]) @ lag for b in range(2)] for a in range(2)])
    return Lg, T


def test_product_rule_matches_graded_rule():
    P, cut, levels = 64, (4,), (5,)
    a, b = X.panels(P, cut, levels)
    nd = X.nodes("star", STAR, a, b)
    coarse_left, fine0 = 3, 4                       # refined order: panel 3, then 32 fine panels
    pairs = [(16 * coarse_left + 15, fine0), (16 * coarse_left + 15, coarse_left),
             (16 * fine0, coarse_left), (16 * fine0 + 3, fine0), (16 * (fine0 + 1) + 8, coarse_left),
             (16 * 20 + 7, 20), (16 * 20 + 15, 21)]
    worst = 0.0
    for i, p in pairs:
        tm, th = 0.5 * (a[p] + b[p]), 0.5 * (b[p] - a[p])
        loc = (np.remainder(nd["t"][i] - tm + np.pi, 2.0 * np.pi) - np.pi) / th
        assert abs(loc) < 2.0
        Lg, T = _product_rule(nd["x"][i], nd["y"][i], loc, tm, th)
        Lo, To = X._near_single_layer("star", STAR, nd, i, a[p], b[p])
        worst = max(worst, np.abs(Lg - Lo).max() / np.abs(Lo).max(), np.abs(T - To).max() / np.abs(To).max())
    assert worst < 1e-11, worst
