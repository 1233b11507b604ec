"""Several refined regions grouped in one refinement (Sec. 5.3, the Remark on
grouping the refined regions of consecutive time steps into one refined
discretisation that shares one factorisation of Q).

Each region (a contiguous run of cut panels) gets its own P^div and P^bas
circles; the far wall rows are compressed against the union of the P^bas
circles and A_pk region by region.  The result must be the solution of the
refined system on the union of the refinements, which the oracle assembles
densely (Sec. 2, Eq. interior_BIE_discretized2) and solves by LU:
* star wall, two windows at different levels (one wrapping past t = 0):
  RW_MODE_DIRECT_REFINED density <= 1e-10, RW_MODE_DIRECT <= 1e-9, and the
  interior velocity against the closed-form Stokeslet field;
* 512-panel channel with op_tol 1e-14, the windows of two consecutive steps of
  the moving schedule grouped, 8 RHS: RW_MODE_DIRECT_IR and
  RW_MODE_GMRES_MIXED certified residual <= 1e-10 against the dense operator;
* the grouped refinement equals, on each snapshot's data, the oracle's
  solution on the grouped discretisation (one factorisation, two snapshots).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import rwsolve, inputs  # noqa: E402
from oracle import discretize as D, stokes as S, dense as DN  # noqa: E402

pytestmark = pytest.mark.gpu
STAR = dict(a=0.3, k=5)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return rwsolve.load(build_if_missing=True)


def test_two_regions_star(lib):
    w = rwsolve.Wall("star", 64, (0.3, 5, 1.0))
    panels = [62, 63, 0, 1, 30, 31, 32]        # a wrap-around window and a second one
    levels = [3, 3, 3, 3, 2, 2, 2]
    r = w.refine(panels, levels)
    st = r.stats()
    sx, sy, f = inputs.stokeslets_star(4, nrhs=2)
    src = np.ascontiguousarray(np.stack([sx, sy], 1))
    fd = np.ascontiguousarray(np.transpose(f, (2, 0, 1)))
    g = np.empty((2, 2 * st["n_n"]))
    r.stokeslet_data(src, fd, g, nrhs=2)
    o = D.refine("star", STAR, 64, panels, levels)
    g_or = S.boundary_data(o["n"], sx, sy, f)
    assert np.abs(g_or.T - g).max() <= 1e-13 * np.abs(g_or).max()
    tau_or = DN.solve_refined(o, g_or)
    tx, ty = inputs.targets_star(6, 10)
    tg = np.ascontiguousarray(np.stack([tx, ty], 1))
    for mode, bar in ((rwsolve.MODE_DIRECT_REFINED, 1e-10), (rwsolve.MODE_DIRECT, 1e-9)):
        tau = np.empty_like(g)
        u = np.empty((2, 2 * tx.size))
        r.solve(g, tau, nrhs=2, targets=tg, u=u, mode=mode)
        err = np.linalg.norm(tau.T - tau_or, axis=0) / np.linalg.norm(tau_or, axis=0)
        print(f"two regions, mode {mode}: density {err.max():.2e}, k = {st['k']}")
        assert err.max() <= bar
        ue = S.stokeslet_velocity(tx, ty, sx, sy, f)
        uu = u.reshape(2, -1, 2).transpose(1, 2, 0)
        assert np.abs(uu - ue).max() <= 1e-8 * np.abs(ue).max()
    r.close()
    w.close()


def test_grouped_consecutive_steps_channel(lib):
    P = 512
    sched = inputs.time_schedule(31, P, 40)
    (p0, l0), (p1, l1) = sched[0], sched[20]          # two windows far apart on the wall
    panels, levels = p0 + p1, l0 + l1
    w = rwsolve.Wall("channel", P, opts=rwsolve.default_opts(op_tol=1e-14))
    r = w.refine(panels, levels)
    st = r.stats()
    o = D.refine("channel", {}, P, panels, levels)
    A = S.matrix(o["n"])
    nrhs = 8
    for snap in (0, 1):                               # the two snapshots share the factorisation
        sx, sy, f = inputs.stokeslet_pairs_channel(50 + snap, nrhs)
        src = np.ascontiguousarray(np.stack([sx, sy], 1))
        fd = np.ascontiguousarray(np.transpose(f, (2, 0, 1)))
        g = np.empty((nrhs, 2 * st["n_n"]))
        r.stokeslet_data(src, fd, g, nrhs=nrhs)
        g_or = S.boundary_data(o["n"], sx, sy, f)
        tau_or = DN.solve_refined(o, g_or)
        for mode in (rwsolve.MODE_DIRECT_IR, rwsolve.MODE_GMRES_MIXED):
            tau = np.empty_like(g)
            info = r.solve(g, tau, nrhs=nrhs, mode=mode)
            res = A @ tau.T - g_or
            rres = (np.linalg.norm(res, axis=0) / np.linalg.norm(g_or, axis=0)).max()
            err = (np.linalg.norm(tau.T - tau_or, axis=0) / np.linalg.norm(tau_or, axis=0)).max()
            print(f"snapshot {snap}, mode {mode}: residual {rres:.2e}, density {err:.2e}, k = {st['k']}")
            assert info["rel_residual"] <= 1e-10
            assert rres <= 1e-10
            assert err <= 1e-7
    r.close()
    w.close()
