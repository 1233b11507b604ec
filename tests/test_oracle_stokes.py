"""Pins for oracle/stokes.py and oracle/dense.py (Sec. 2, Sec. 3.2-3.4).

* unit circle, constant data: tau = -g exactly (the circle's double-layer
  kernel is a trigonometric polynomial, integrated exactly by the panels);
* left null vector of -1/2 I + D and the N correction (Remark 2.1):
  (w (x) n)^T A = |Gamma| (w (x) n)^T;
* consistency of Stokeslet data, int g . n ds = 0 (Sec. 2.1);
* closed form: the interior velocity of the solved density equals the
  Stokeslet field that made the data (Sec. 5 preamble), with spectral decay
  of the error under panel refinement;
* closed form for the pressure: the double-layer pressure of the solved
  density equals the Stokeslet pressure up to one constant (pressure is
  fixed up to a constant by the velocity), with spectral decay; a sign error
  in either term of the pressure kernel breaks the constant offset;
* the row-at-a-time residual agrees with the dense matrix;
* ELS equivalence (Eq. extendedlLinearSystem), Woodbury exactness for Q = L R
  (Eq. wood), truncated-SVD Woodbury accuracy, Lemma 3.1's bound, and the
  rank drop of the recompression (Sec. 3.4, Tab. conditiontest)."""
import numpy as np
import pytest

from oracle import discretize as D, stokes as S, dense as DN
from paper_2108_07205_gb300 import inputs as I

STAR = dict(a=0.3, k=5)


def _wn(nodes):
    v = np.zeros(2 * nodes["x"].size)
    v[0::2] = nodes["w"] * nodes["nx"]
    v[1::2] = nodes["w"] * nodes["ny"]
    return v


@pytest.mark.parametrize("panels", [4, 8])
def test_circle_constant_density(panels):
    n = D.wall_nodes("star", dict(a=0.0, k=1), panels)
    A = S.matrix(n)
    g = np.tile([0.3, -0.7], n["x"].size)
    tau = np.linalg.solve(A, g)
    assert np.abs(tau + g).max() < 1e-13


@pytest.mark.parametrize("kind,params,P", [("star", STAR, 32), ("channel", {}, 128)])
def test_left_null_vector_and_N(kind, params, P):
    n = D.wall_nodes(kind, params, P)
    A = S.matrix(n)
    wn = _wn(n)
    perim = n["w"].sum()
    assert np.abs(wn @ A - perim * wn).max() < 1e-12 * perim
    # without N the same vector annihilates -1/2 I + D
    A0 = A - np.outer(np.ravel(np.stack([n["nx"], n["ny"]], 1)), wn)
    assert np.abs(wn @ A0).max() < 1e-12


def test_stokeslet_data_is_consistent():
    n = D.wall_nodes("star", STAR, 32)
    sx, sy, f = I.stokeslets_star(3, nrhs=4)
    g = S.boundary_data(n, sx, sy, f)
    assert np.abs(_wn(n) @ g).max() < 1e-13


def _closed_form_error(nodes, sx, sy, f, tx, ty):
    A = S.matrix(nodes)
    g = S.boundary_data(nodes, sx, sy, f)
    tau = np.linalg.solve(A, g)
    u = S.velocity(nodes, tau, tx, ty)
    ue = S.stokeslet_velocity(tx, ty, sx, sy, f)
    return np.abs(u - ue).max() / np.abs(ue).max(), tau, g


def test_closed_form_and_spectral_convergence_star():
    sx, sy, f = I.stokeslets_star(0, nrhs=2)
    tx, ty = I.targets_star(1)
    errs = [_closed_form_error(D.wall_nodes("star", STAR, P), sx, sy, f, tx, ty)[0]
            for P in (8, 12, 16, 64)]
    assert errs[-1] < 1e-12
    assert errs[0] > errs[1] > errs[2]
    # integral of tau . n vanishes for consistent data
    _, tau, _ = _closed_form_error(D.wall_nodes("star", STAR, 32), sx, sy, f, tx, ty)
    assert np.abs(_wn(D.wall_nodes("star", STAR, 32)) @ tau).max() < 1e-12


def test_closed_form_channel():
    n = D.wall_nodes("channel", {}, 256)
    sx, sy, f = I.stokeslets_channel(0)
    tx, ty = I.targets_channel(1)
    err = _closed_form_error(n, sx, sy, f, tx, ty)[0]
    assert err < 1e-9


def test_closed_form_refined_star():
    ref = D.refine("star", STAR, 64, [62, 63, 0, 1], [3] * 4)
    sx, sy, f = I.stokeslets_star(0, nrhs=2)
    tx, ty = I.targets_star(1)
    g = S.boundary_data(ref["n"], sx, sy, f)
    tau = DN.solve_refined(ref, g)
    u = S.velocity(ref["n"], tau, tx, ty)
    ue = S.stokeslet_velocity(tx, ty, sx, sy, f)
    assert np.abs(u - ue).max() / np.abs(ue).max() < 1e-12


def _pressure_offset_spread(nodes, sx, sy, f, tx, ty, kernel=None):
    """Spread of p_DLP(tau) - p_exact over the targets, relative to the
    spread of p_exact (zero when they differ by one constant)."""
    g = S.boundary_data(nodes, sx, sy, f)
    tau = np.linalg.solve(S.matrix(nodes), g)
    p = (kernel or S.pressure)(nodes, tau, tx, ty)
    pe = S.stokeslet_pressure(tx, ty, sx, sy, f)
    diff = p - pe
    return np.abs(diff - diff.mean(axis=0)).max() / np.abs(pe - pe.mean(axis=0)).max()


def test_pressure_closed_form_up_to_a_constant():
    sx, sy, f = I.stokeslets_star(0, nrhs=2)
    tx, ty = I.targets_star(1)
    spreads = [_pressure_offset_spread(D.wall_nodes("star", STAR, P), sx, sy, f, tx, ty) for P in (8, 16, 64)]
    assert spreads[-1] < 1e-11
    assert spreads[0] > spreads[1] > spreads[2]
    # refined wall: the refined density's pressure meets the same closed form
    ref = D.refine("star", STAR, 64, [62, 63, 0, 1], [3] * 4)
    tau = DN.solve_refined(ref, S.boundary_data(ref["n"], sx, sy, f))
    dp = S.pressure(ref["n"], tau, tx, ty) - S.stokeslet_pressure(tx, ty, sx, sy, f)
    assert np.abs(dp - dp.mean(axis=0)).max() < 1e-10


def test_pressure_pins_catch_sign_errors():
    n = D.wall_nodes("star", STAR, 64)
    sx, sy, f = I.stokeslets_star(0, nrhs=1)
    tx, ty = I.targets_star(1)

    def flipped(which):
        def k(nodes, tau, tx_, ty_):
            # the same sum with one term's sign flipped (a planted mistake)
            tau = np.asarray(tau)[:, None] if np.ndim(tau) == 1 else np.asarray(tau)
            rx = np.asarray(tx_)[:, None] - nodes["x"][None, :]
            ry = np.asarray(ty_)[:, None] - nodes["y"][None, :]
            r2 = rx * rx + ry * ry
            rdn = rx * nodes["nx"][None, :] + ry * nodes["ny"][None, :]
            ndt = nodes["nx"][None, :, None] * tau[0::2][None] + nodes["ny"][None, :, None] * tau[1::2][None]
            rdt = rx[:, :, None] * tau[0::2][None] + ry[:, :, None] * tau[1::2][None]
            a = -ndt / r2[:, :, None]
            b = 2.0 * rdt * rdn[:, :, None] / (r2 * r2)[:, :, None]
            s = (-a + b) if which == 0 else (a - b)
            return np.sum(nodes["w"][None, :, None] * s, axis=1)[:, 0] / np.pi
        return k

    assert _pressure_offset_spread(n, sx, sy, f, tx, ty) < 1e-11
    for which in (0, 1):
        assert _pressure_offset_spread(n, sx, sy, f, tx, ty, flipped(which)) > 1e-3


def test_apply_rows_matches_matrix():
    n = D.wall_nodes("star", STAR, 8)
    A = S.matrix(n)
    tau = I.rng(5).standard_normal((A.shape[0], 3))
    rows = [0, 1, 17, 64, A.shape[0] - 1]
    assert np.abs(S.apply_rows(n, tau, rows) - (A @ tau)[rows]).max() < 1e-14


def _tiny():
    ref = D.refine("star", STAR, 12, [3, 4], [2, 2])
    sx, sy, f = I.stokeslets_star(0, nrhs=2)
    g_n = S.boundary_data(ref["n"], sx, sy, f)
    return ref, g_n


def test_extended_system_equivalence():
    ref, g_n = _tiny()
    ext = DN.extended_system(ref)
    assert np.allclose(ext["A_ext"], ext["At"] + ext["Q"], atol=0)
    tau_ext = np.linalg.solve(ext["A_ext"], DN.g_ext(ref, g_n))
    tau_n = DN.solve_refined(ref, g_n)
    assert np.abs(DN.ext_to_n(ref, tau_ext) - tau_n).max() < 1e-12 * np.abs(tau_n).max()


def test_woodbury_exact_and_svd():
    ref, g_n = _tiny()
    ext = DN.extended_system(ref)
    g = DN.g_ext(ref, g_n)
    tau_n = DN.solve_refined(ref, g_n)
    scale = np.abs(tau_n).max()
    # exact factors: L = Q's nonzero columns, R = selector of those columns
    cols = np.where(np.abs(ext["Q"]).sum(0) > 0)[0]
    L = ext["Q"][:, cols]
    R = np.zeros((cols.size, ext["Q"].shape[0]))
    R[np.arange(cols.size), cols] = 1.0
    tau_ext, _ = DN.woodbury(ext, L, R, g)
    assert np.abs(DN.ext_to_n(ref, tau_ext) - tau_n).max() < 1e-12 * scale
    for tol, bound in ((1e-8, 1e-6), (1e-12, 1e-10)):
        L, R = DN.svd_factors(ext, tol)
        tau_ext, W = DN.woodbury(ext, L, R, g)
        assert np.abs(DN.ext_to_n(ref, tau_ext) - tau_n).max() < bound * scale


def test_lemma_3_1_bound_and_recompression():
    ref, g_n = _tiny()
    ext = DN.extended_system(ref)
    tol = 1e-10
    Lb, Rb = DN.svd_factors(ext, tol, recompress=False)
    Lo, Ro = DN.svd_factors(ext, tol, recompress=True)
    assert Lo.shape[1] < Lb.shape[1]          # k_optimal < k_block
    for L, R in ((Lb, Rb), (Lo, Ro)):
        X = np.linalg.solve(ext["At"], L)
        W = np.eye(L.shape[1]) + R @ X
        kw = np.linalg.cond(W)
        bound = min(DN.pinv_cond(L) ** 2, DN.pinv_cond(R.T) ** 2) * \
            np.linalg.cond(ext["At"] + L @ R) * np.linalg.cond(ext["At"])
        assert kw <= bound
    # recompressed L has orthonormal columns: kappa-hat(L) = 1
    assert abs(DN.pinv_cond(Lo) - 1.0) < 1e-10
