"""GPU parity of the exterior wall (Sec. 2.2, Eq. exterior_BIE: the fluid
outside the star, combined field 1/2 I + D + S) against oracle/exterior.py.

The GPU integrates the single layer's logarithm near each target by Legendre
product integration on a 32-point auxiliary rule.  The oracle uses a graded
brute-force rule.  Both are exact for the density's panel interpolant to
rounding.  Tolerances (relative 2-norm), from the arithmetic:
* nodes and boundary data: 1e-13.
* Forward HBS apply against the oracle's dense matrix: 1e-11 (compression
  1e-12).  Inverse against the dense solve: 1e-10 (kappa ~ 10).
* Refined density: RW_MODE_DIRECT 1e-10 and RW_MODE_DIRECT_REFINED 1e-11,
  against the oracle's LU of the refined system.  The exact refined apply
  (entries on the fly, with the singular rule) against the dense matrix:
  1e-12.
* The certified modes on walls with op_tol = 1e-14 (RW_MODE_DIRECT_IR,
  RW_MODE_DIRECT_IR_DF, RW_MODE_GMRES_FP32): true residual against the
  oracle's dense refined matrix <= 1e-10 per right-hand side.
* Velocity at points of the fluid against the closed-form field of the
  Stokeslets inside the wall: 1e-10.
* The constricted channel as an exterior wall (128 panels, a refined window):
  density against the oracle's LU and velocity against the oracle's, 1e-10;
  velocity against the closed form 1e-9 (the oracle's own discretisation
  error there is 1.2e-10).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import rwsolve, inputs  # noqa: E402
from oracle import exterior as X, stokes as S  # noqa: E402

pytestmark = pytest.mark.gpu

STAR = dict(a=0.3, k=5)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return rwsolve.load(build_if_missing=True)


@pytest.fixture(scope="module")
def ext64(lib):
    w = rwsolve.Wall("star", 64, (0.3, 5, 1.0), exterior=True)
    yield w
    w.close()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_refined(panels, levels, P=64):
    a, b = X.panels(P, panels, levels)
    return X.nodes("star", STAR, a, b)


def data(ref, nd, seed, nrhs):
    sx, sy, f = inputs.stokeslets_inside_star(seed, nrhs=nrhs)
    src = np.ascontiguousarray(np.stack([sx, sy], 1))
    fd = np.ascontiguousarray(np.transpose(f, (2, 0, 1)))
    g = np.empty((nrhs, 2 * ref.stats()["n_n"]))
    ref.stokeslet_data(src, fd, g, nrhs=nrhs)
    return g, S.boundary_data(nd, sx, sy, f).T, (sx, sy, f)


def test_exterior_wall_matrix_and_inverse(ext64):
    a, b = X.panels(64)
    nd = X.nodes("star", STAR, a, b)
    wn = ext64.nodes()
    for key in ("x", "y", "nx", "ny", "w", "kappa"):
        assert np.abs(wn[key] - nd[key]).max() <= 1e-13 * (1 + np.abs(nd[key]).max()), key
    A = X.matrix("star", STAR, nd)
    x = inputs.rng(4).standard_normal((3, A.shape[0]))
    y = np.empty_like(x)
    ext64.apply_forward(x, y, nrhs=3)
    assert rel(y, (A @ x.T).T) < 1e-11
    z = np.empty_like(x)
    ext64.apply_inverse(x, z, nrhs=3)
    assert rel(z, np.linalg.solve(A, x.T).T) < 1e-10


@pytest.mark.parametrize("panels,levels", [
    (None, None),                          # seeded 4-panel window at level 3
    ([62, 63, 0, 1], [2, 4, 3, 5]),        # wrap-around, ragged levels: HBS of the refined arc
    ([10], [2]),                           # 64 added points: dense A_pp
])
def test_exterior_refined_solve_vs_oracle(ext64, panels, levels):
    if panels is None:
        panels, levels = inputs.refinement_window(7, 64, 4, 3, 3)
    ref = ext64.refine(panels, levels)
    nd = oracle_refined(panels, levels)
    rn = ref.nodes()
    for key in ("x", "y", "nx", "ny", "w", "kappa"):
        assert np.abs(rn[key] - nd[key]).max() <= 1e-13 * (1 + np.abs(nd[key]).max())
    g, g_or, (sx, sy, f) = data(ref, nd, 2, 3)
    assert np.abs(g - g_or).max() <= 1e-13 * np.abs(g_or).max()
    tau_or = X.solve("star", STAR, nd, g_or.T).T
    tx, ty = inputs.targets_outside_star(5)
    tg = np.ascontiguousarray(np.stack([tx, ty], 1))
    u = np.empty((3, 2 * tx.size))
    tau = np.empty_like(g)
    ref.solve(g, tau, nrhs=3, targets=tg, u=u)
    assert rel(tau, tau_or) < 1e-10
    ue = np.transpose(S.stokeslet_velocity(tx, ty, sx, sy, f), (2, 0, 1)).reshape(3, -1)
    assert np.abs(u - ue).max() < 1e-10 * np.abs(ue).max()
    tau_r = np.empty_like(g)
    ref.solve(g, tau_r, nrhs=3, mode=rwsolve.MODE_DIRECT_REFINED)
    assert rel(tau_r, tau_or) < 1e-11
    ref.close()


def test_exterior_exact_apply_vs_dense(ext64):
    panels, levels = [20, 21, 22], [3, 2, 3]
    ref = ext64.refine(panels, levels)
    A = X.matrix("star", STAR, oracle_refined(panels, levels))
    t = inputs.rng(6).standard_normal((2, A.shape[0]))
    y = np.empty_like(t)
    ref.apply_refined(t, y, nrhs=2)
    assert rel(y, (A @ t.T).T) < 1e-12
    ref.close()


def test_exterior_two_regions(ext64):
    panels, levels = [5, 6, 7, 40, 41], [3, 3, 3, 2, 4]
    ref = ext64.refine(panels, levels)
    nd = oracle_refined(panels, levels)
    g, g_or, _ = data(ref, nd, 8, 2)
    tau = np.empty_like(g)
    ref.solve(g, tau, nrhs=2)
    assert rel(tau, X.solve("star", STAR, nd, g_or.T).T) < 1e-10
    ref.close()


@pytest.mark.parametrize("mode,mixed_factor", [
    (rwsolve.MODE_DIRECT_IR, 0), (rwsolve.MODE_DIRECT_IR_DF, 2), (rwsolve.MODE_GMRES_FP32, 0)])
def test_exterior_certified_modes(lib, mode, mixed_factor):
    w = rwsolve.Wall("star", 64, (0.3, 5, 1.0), exterior=True,
                     opts=rwsolve.default_opts(op_tol=1e-14, mixed_factor=mixed_factor))
    panels, levels = inputs.refinement_window(9, 64, 4, 4, 4)
    ref = w.refine(panels, levels)
    nd = oracle_refined(panels, levels)
    nrhs = 12
    g, g_or, _ = data(ref, nd, 10, nrhs)
    tau = np.empty_like(g)
    info = ref.solve(g, tau, nrhs=nrhs, mode=mode)
    assert info["rel_residual"] <= 1e-10
    A = X.matrix("star", STAR, nd)
    for r in range(nrhs):
        res = np.linalg.norm(g_or[r] - A @ tau[r]) / np.linalg.norm(g_or[r])
        assert res <= 1e-10, (r, res)
    assert rel(tau, np.linalg.solve(A, g_or.T).T) < 1e-10
    ref.close()
    w.close()


def test_exterior_channel_vs_oracle(lib):
    # the constricted channel as an exterior wall (128 panels), a refined
    # window at level 3: density against the oracle's LU, velocity outside
    # the channel against the closed form
    panels, levels = [40, 41, 42, 43], [3, 3, 3, 3]
    w = rwsolve.Wall("channel", 128, exterior=True)
    ref = w.refine(panels, levels)
    a, b = X.panels(128, panels, levels)
    nd = X.nodes("channel", {}, a, b)
    sx, sy, f = inputs.stokeslets_inside_channel(11, nrhs=2)
    src = np.ascontiguousarray(np.stack([sx, sy], 1))
    fd = np.ascontiguousarray(np.transpose(f, (2, 0, 1)))
    g = np.empty((2, 2 * ref.stats()["n_n"]))
    ref.stokeslet_data(src, fd, g, nrhs=2)
    g_or = S.boundary_data(nd, sx, sy, f).T
    assert np.abs(g - g_or).max() <= 1e-13 * np.abs(g_or).max()
    tx, ty = inputs.targets_outside_channel(12)
    tg = np.ascontiguousarray(np.stack([tx, ty], 1))
    u = np.empty((2, 2 * tx.size))
    tau = np.empty_like(g)
    ref.solve(g, tau, nrhs=2, targets=tg, u=u)
    tau_or = X.solve("channel", {}, nd, g_or.T).T
    assert rel(tau, tau_or) < 1e-10
    uo = np.transpose(X.velocity(nd, tau_or.T, tx, ty), (2, 0, 1)).reshape(2, -1)
    assert np.abs(u - uo).max() < 1e-10 * np.abs(uo).max()
    # 128 panels resolve these sources (0.1 from a wall 0.2 away) to 1.2e-10
    # in the oracle itself
    ue = np.transpose(S.stokeslet_velocity(tx, ty, sx, sy, f), (2, 0, 1)).reshape(2, -1)
    assert np.abs(u - ue).max() < 1e-9 * np.abs(ue).max()
    ref.close()
    w.close()


def test_exterior_refusals(ext64, tmp_path):
    with pytest.raises(rwsolve.RWError):
        ext64.save(str(tmp_path / "ext.rwh"))
    with pytest.raises(rwsolve.RWError):
        ext64.add_holes([dict(cx=0.0, cy=0.0, R=0.1, a=0.0, k=1, P=10)])
    with pytest.raises(rwsolve.RWError):
        rwsolve.Wall("star", 4, (0.3, 5, 1.0), exterior=True)
