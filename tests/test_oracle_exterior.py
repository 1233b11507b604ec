"""Pins for oracle/exterior.py: the exterior Stokes problem on one wall
(Sec. 2.2, Eq. exterior_BIE), reference and locally refined.

* Closed form.  For data made by Stokeslets inside the curve, the combined
  field of the solved density equals the Stokeslet field at points of the
  fluid.  The decay is spectral under panel refinement.  This holds on the
  reference star and on refined stars, where fine panels sit next to coarse
  ones, and outside the constricted channel.
* Total force.  The density's total force sum_j w_j tau_j equals the
  Stokeslets' total force.
* On one equal-panel curve the matrix equals oracle/holes.py's hole matrix,
  which the Fourier closed forms pin.
* The refined order of the panels is the interior wall's (discretize.refine).
* Planted mistakes break the closed form: the interior jump -1/2, the plain
  rule on the log singularity, and a sign flip of the single layer.
* The extended linear system of Sec. 3.2 assembled from the exterior
  operator gives the refined exterior solve, and so does the Woodbury formula
  with exact factors of Q and with truncated-SVD factors within their
  tolerance (the Remark closing Sec. 3.1).
"""
import numpy as np
import pytest

from oracle import exterior as X, holes as H, discretize as D
from paper_2108_07205_gb300 import inputs as I

STAR = dict(a=0.3, k=5)


def _field_error(P, cut=(), levels=(), seed=3):
    a, b = X.panels(P, cut, levels)
    nd = X.nodes("star", STAR, a, b)
    sx, sy, f = I.stokeslets_inside_star(seed, nrhs=2)
    from oracle import stokes as S
    g = S.boundary_data(nd, sx, sy, f)
    tau = X.solve("star", STAR, nd, g)
    tx, ty = I.targets_outside_star(seed + 1, n=12)
    u = X.velocity(nd, tau, tx, ty)
    ue = S.stokeslet_velocity(tx, ty, sx, sy, f)
    return np.abs(u - ue).max() / np.abs(ue).max(), nd, tau, f


def test_closed_form_and_spectral_decay():
    errs = [_field_error(P)[0] for P in (12, 16, 24)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-12
    assert errs[0] > 1e-9   # the coarse mesh is visibly under-resolved: the pin has teeth


@pytest.mark.parametrize("cut,levels", [((5, 6, 7), (3, 3, 3)), ((23, 0, 1), (2, 4, 3))])
def test_closed_form_refined(cut, levels):
    err = _field_error(24, cut, levels)[0]
    assert err < 1e-11


def test_closed_form_outside_the_channel():
    # the constricted 20 x 1 channel as an exterior wall: 128 panels, and the
    # same with a refined window
    from oracle import stokes as S
    sx, sy, f = I.stokeslets_inside_channel(4, nrhs=2)
    tx, ty = I.targets_outside_channel(5, n=12)
    ue = S.stokeslet_velocity(tx, ty, sx, sy, f)
    for cut, levels in (((), ()), ((10, 11, 12), (3, 3, 3))):
        a, b = X.panels(128, cut, levels)
        nd = X.nodes("channel", {}, a, b)
        tau = X.solve("channel", {}, nd, S.boundary_data(nd, sx, sy, f))
        u = X.velocity(nd, tau, tx, ty)
        assert np.abs(u - ue).max() < 1e-10 * np.abs(ue).max()


def test_total_force_identity():
    _, nd, tau, f = _field_error(24, (2, 3), (3, 3))
    F = X.total_force(nd, tau)
    Fs = f.sum(axis=0)
    assert np.abs(F - Fs).max() < 1e-11 * np.abs(Fs).max()


def test_matches_pinned_hole_matrix():
    P = 12
    a, b = X.panels(P)
    nd = X.nodes("star", STAR, a, b)
    A = X.matrix("star", STAR, nd)
    hl = [dict(cx=0.0, cy=0.0, R=1.0, a=STAR["a"], k=STAR["k"], P=P)]
    hn = H.hole_nodes(hl)
    assert np.abs(hn["x"] - nd["x"]).max() < 1e-14
    Ah = H.hole_matrix(hn, hl, 0.5)
    assert np.abs(A - Ah).max() < 1e-13 * np.abs(Ah).max()


def test_refined_order_is_the_interior_walls():
    P, cut, levels = 16, (15, 0, 1), (2, 3, 2)
    a, b = X.panels(P, cut, levels)
    nd = X.nodes("star", STAR, a, b)
    ref = D.refine("star", STAR, P, list(cut), list(levels))
    for key in ("x", "y", "w", "nx", "ny", "kappa"):
        assert np.abs(nd[key] - ref["n"][key]).max() < 1e-13


def test_near_panels_cover_the_refinement_boundary():
    # the coarse nodes closest to a fine run take the graded rule on the fine
    # panel beside them, and every fine node of that run on the coarse panel
    P, cut, levels = 16, (4,), (4,)
    a, b = X.panels(P, cut, levels)
    nd = X.nodes("star", STAR, a, b)
    coarse_left, fine_first = 3, 4
    for i in range(16 * coarse_left + 13, 16 * (coarse_left + 1)):
        assert fine_first in X.near_panels(nd, i)
    assert fine_first not in X.near_panels(nd, 16 * coarse_left)
    for i in range(16 * fine_first, 16 * (fine_first + 16)):
        assert coarse_left in X.near_panels(nd, i)


def test_planted_mistakes_break_the_closed_form(monkeypatch):
    base = _field_error(24)[0]
    assert base < 1e-12
    with monkeypatch.context() as m:
        m.setattr(X, "JUMP", -0.5)
        assert _field_error(24)[0] > 1e-3
    with monkeypatch.context() as m:
        m.setattr(X, "NEAR_LOC", 0.0)
        assert _field_error(24)[0] > 1e-6
    with monkeypatch.context() as m:
        sl = X.single_layer_matrix
        m.setattr(X, "single_layer_matrix", lambda *a: -sl(*a))
        assert _field_error(24)[0] > 1e-3


def test_extended_system_and_woodbury_exterior():
    from oracle import dense as DN, stokes as S
    P, cut, levels = 12, (3, 4), (2, 2)
    ext = X.extended_system("star", STAR, P, cut, levels)
    ref = ext["ref"]
    a, b = X.panels(P, cut, levels)
    nd = X.nodes("star", STAR, a, b)
    for key in ("x", "y", "w"):
        assert np.abs(nd[key] - ref["n"][key]).max() < 1e-13
    sx, sy, f = I.stokeslets_inside_star(6, nrhs=2)
    g_n = S.boundary_data(nd, sx, sy, f)
    tau_n = X.solve("star", STAR, nd, g_n)
    scale = np.abs(tau_n).max()
    g = DN.g_ext(ref, g_n)
    tau_ext = np.linalg.solve(ext["A_ext"], g)
    assert np.abs(DN.ext_to_n(ref, tau_ext) - tau_n).max() < 1e-12 * scale
    cols = np.where(np.abs(ext["Q"]).sum(0) > 0)[0]
    L = ext["Q"][:, cols]
    R = np.zeros((cols.size, ext["Q"].shape[0]))
    R[np.arange(cols.size), cols] = 1.0
    tau_w, _ = DN.woodbury(ext, L, R, g)
    assert np.abs(DN.ext_to_n(ref, tau_w) - tau_n).max() < 1e-12 * scale
    for tol, bound in ((1e-8, 1e-6), (1e-12, 1e-10)):
        L, R = DN.svd_factors(ext, tol)
        tau_w, _ = DN.woodbury(ext, L, R, g)
        assert np.abs(DN.ext_to_n(ref, tau_w) - tau_n).max() < bound * scale
