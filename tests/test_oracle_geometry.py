"""Pins for oracle/quadrature.py, oracle/curves.py and oracle/discretize.py.

Checks against closed forms and brute force (Sec. 3.1, Sec. 5 preamble):
exact polynomial integration of the 16-point rule, the star's enclosed area
pi (1 + a^2 / 2), total curvature 2 pi of a simple closed curve, the channel's
area against a shoelace polygon, derivatives against finite differences, and
the bookkeeping of local refinement (weights, ordering, index sets)."""
import numpy as np
import pytest

from oracle import curves, discretize as D
from oracle.quadrature import gauss_legendre


def test_gauss_legendre_exact_to_degree_31():
    x, w = gauss_legendre(16)
    assert x.size == 16 and np.all(np.diff(x) > 0)
    for d in range(32):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) < 1e-14
    # degree 32 is not integrated exactly by a 16-point rule
    assert abs(np.sum(w * x ** 32) - 2.0 / 33) > 1e-12


@pytest.mark.parametrize("a,k", [(0.0, 1), (0.3, 5), (0.2, 3)])
def test_star_area_perimeter_curvature(a, k):
    n = D.wall_nodes("star", dict(a=a, k=k), 64)
    area = 0.5 * np.sum(n["w"] * (n["x"] * n["nx"] + n["y"] * n["ny"]))
    assert abs(area - np.pi * (1 + a * a / 2)) < 1e-13
    assert abs(np.sum(n["kappa"] * n["w"]) - 2 * np.pi) < 1e-12
    if a == 0.0:
        assert abs(n["w"].sum() - 2 * np.pi) < 1e-13
        assert np.allclose(n["kappa"], 1.0, atol=1e-14)
        # outward normal of the unit circle is the position vector
        assert np.allclose(n["nx"], n["x"], atol=1e-15)
        assert np.allclose(n["ny"], n["y"], atol=1e-15)


def test_channel_area_and_curvature():
    n = D.wall_nodes("channel", {}, 512)
    area = 0.5 * np.sum(n["w"] * (n["x"] * n["nx"] + n["y"] * n["ny"]))
    t = np.linspace(0, 2 * np.pi, 400001)[:-1]
    g = curves.evaluate("channel", t)
    x, y = g["x"], g["y"]
    shoelace = 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)
    assert abs(area - shoelace) < 1e-6 * shoelace
    assert abs(np.sum(n["kappa"] * n["w"]) - 2 * np.pi) < 1e-10
    # the constriction: half-height 0.2 at x = 0, about 0.5 near the ends
    top = curves.evaluate("channel", np.array([np.pi / 2]))
    assert abs(top["y"][0] - 0.2) < 1e-14 and abs(top["x"][0]) < 1e-14


@pytest.mark.parametrize("kind,params", [("star", dict(a=0.3, k=5)), ("channel", {})])
def test_derivatives_match_finite_differences(kind, params):
    t = np.linspace(0.1, 6.1, 37)
    h = 1e-4
    g0 = curves.evaluate(kind, t, **params)
    gp = curves.evaluate(kind, t + h, **params)
    gm = curves.evaluate(kind, t - h, **params)
    for c in "xy":
        fd1 = (gp[c] - gm[c]) / (2 * h)
        fd2 = (gp[c] - 2 * g0[c] + gm[c]) / h ** 2
        scale = 1 + np.abs(g0["d" + c]).max()
        assert np.abs(fd1 - g0["d" + c]).max() < 1e-6 * scale
        assert np.abs(fd2 - g0["dd" + c]).max() < 1e-3 * (1 + np.abs(g0["dd" + c]).max())


@pytest.mark.parametrize("panels,levels", [([5, 6, 7, 8], [3] * 4), ([62, 63, 0, 1], [2, 3, 1, 2])])
def test_refinement_bookkeeping(panels, levels):
    P = 64
    ref = D.refine("star", dict(a=0.3, k=5), P, panels, levels)
    o, p, n = ref["o"], ref["p"], ref["n"]
    assert ref["I_k"].size + ref["I_c"].size == o["x"].size
    assert np.intersect1d(ref["I_k"], ref["I_c"]).size == 0
    assert p["x"].size == 16 * sum(2 ** L for L in levels)
    assert n["x"].size == ref["I_k"].size + p["x"].size
    # same curve, same total length and integral of x n_x (area) to rounding
    for key in ("w",):
        assert abs(n[key].sum() - o[key].sum()) < 1e-13
    area_o = 0.5 * np.sum(o["w"] * (o["x"] * o["nx"] + o["y"] * o["ny"]))
    area_n = 0.5 * np.sum(n["w"] * (n["x"] * n["nx"] + n["y"] * n["ny"]))
    assert abs(area_o - area_n) < 1e-13
    # refined order is increasing in t; added points in window order
    assert np.all(np.diff(n["t"]) > 0)
    starts = [p["t"][16 * sum(2 ** L for L in levels[:i])] for i in range(len(levels))]
    h = 2 * np.pi / P
    for j, t0 in zip(panels, starts):
        assert j * h < t0 < (j + 1) * h
