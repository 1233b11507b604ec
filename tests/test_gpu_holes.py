"""Oracle parity of the wall with added holes (App. B) through the C ABI.

* the exact operator A_nn (rw_apply_refined) against the oracle's dense
  system, entry by entry through random vectors, with the paper's circles
  and with star-shaped holes: the holes' combined field with its singular
  rule (Legendre product integration on a 32-point auxiliary rule here,
  graded Gauss there, both exact for the density's interpolant), the cross
  blocks and the wall block, <= 1e-13 relative;
* densities from the three solve modes against the oracle's dense LU solve
  on the star wall with circular and star-shaped holes and on the channel:
  RW_MODE_DIRECT_REFINED at <= 1e-10 relative (the FP64 parity bar),
  RW_MODE_DIRECT at <= 1e-8 (one compressed solve: 1e-12 IDs times the
  conditioning of the holed system); FGMRES, which stops on the residual of
  the compressed (ELS) operator: that residual <= 1e-10 (as for the refined
  channel), the residual of the oracle's dense operator <= 1e-9 (the ELS
  operator carries the 1e-12 compression) and the density within 1e-10
  times the oracle's condition estimate of A_nn;
* the velocity and pressure in the fluid against the oracle's evaluation and
  the closed-form Stokeslet field;
* on the 1024-panel channel with the paper's three holes of 10 panels
  (Sec. 5.2), too large for a dense oracle solve: 32 sampled residual rows
  of the exact operator, each written out by the oracle, and the closed-form
  velocity;
* invalid hole layouts are rejected with RW_ERR_INVALID.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import rwsolve, inputs  # noqa: E402
from oracle import discretize as D, stokes as S, holes as H  # noqa: E402

pytestmark = pytest.mark.gpu
STAR = dict(a=0.3, k=5)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return rwsolve.load(build_if_missing=True)


def _case(kind, P, PH, hole_a=0.0, hole_k=1, nrhs=2):
    if kind == "star":
        wall_o = D.wall_nodes("star", STAR, P)
        hl = inputs.holes_star(3, n_panels=PH, a=hole_a, k=hole_k)
        sx, sy, f = inputs.stokeslets_star(0, nrhs=nrhs)
        w = rwsolve.Wall("star", P, (0.3, 5, 1.0))
    else:
        wall_o = D.wall_nodes("channel", {}, P)
        hl = inputs.holes_channel(3, n_panels=PH)
        sx, sy, f = inputs.stokeslets_channel(0, nrhs=nrhs)
        w = rwsolve.Wall("channel", P)
    hx, hy, hf = inputs.stokeslets_in_holes(1, hl, [2, 2, 1], nrhs=nrhs)
    src = (np.concatenate([sx, hx]), np.concatenate([sy, hy]), np.concatenate([f, hf]))
    return w, wall_o, hl, src


def _device_data(r, src, nrhs):
    sx, sy, f = src
    g = np.empty((nrhs, 2 * r.stats()["n_n"]))
    r.stokeslet_data(np.ascontiguousarray(np.stack([sx, sy], 1)), np.ascontiguousarray(np.transpose(f, (2, 0, 1))),
                     g, nrhs=nrhs)
    return g


@pytest.mark.parametrize("PH,a,k", [(10, 0.0, 1), (12, 0.2, 3)])
def test_operator_matches_oracle(lib, PH, a, k):
    w, wall_o, hl, src = _case("star", 24, PH, hole_a=a, hole_k=k)
    r = w.add_holes(hl)
    hn = H.hole_nodes(hl)
    A = H.system(wall_o, hn, hl)
    st = r.stats()
    assert st["n_c"] == 0 and st["n_p"] == hn["x"].size and st["n_n"] == A.shape[0] // 2
    nodes = r.nodes()
    xy = np.concatenate([wall_o["x"], hn["x"]]), np.concatenate([wall_o["y"], hn["y"]])
    assert np.abs(nodes["x"] - xy[0]).max() < 1e-14 and np.abs(nodes["y"] - xy[1]).max() < 1e-14
    x = inputs.rng(11).standard_normal((3, A.shape[0]))
    y = np.empty_like(x)
    r.apply_refined(x, y, nrhs=3)
    ref = (A @ x.T).T
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    # the hole block alone (where the two singular rules differ)
    nk = 2 * wall_o["x"].size
    xh = np.zeros_like(x)
    xh[:, nk:] = x[:, nk:]
    r.apply_refined(xh, y, nrhs=3)
    ref = (A @ xh.T).T
    assert np.abs(y[:, nk:] - ref[:, nk:]).max() <= 1e-13 * np.abs(ref[:, nk:]).max()
    r.close()
    w.close()


@pytest.mark.parametrize("kind,P,PH,a,k", [("star", 32, 6, 0.0, 1), ("star", 32, 12, 0.2, 3), ("channel", 256, 10, 0.0, 1)])
def test_solve_modes_match_oracle(lib, kind, P, PH, a, k):
    nrhs = 2
    w, wall_o, hl, src = _case(kind, P, PH, a, k, nrhs)
    r = w.add_holes(hl)
    hn = H.hole_nodes(hl)
    g = _device_data(r, src, nrhs)
    g_or = H.boundary_data(wall_o, hn, *src)
    assert np.abs(g - g_or.T).max() <= 1e-13 * np.abs(g_or).max()
    A_or = H.system(wall_o, hn, hl)
    tau_or = np.linalg.solve(A_or, g_or).T
    nrm = np.linalg.norm(tau_or, axis=1)
    kappa = np.linalg.cond(A_or)
    tg = inputs.targets_fluid(2, hl, kind, 12)
    ue = S.stokeslet_velocity(*tg, *src)                                  # (nt, 2, nrhs)
    for mode, bar in ((rwsolve.MODE_DIRECT_REFINED, 1e-10), (rwsolve.MODE_GMRES_FP32, 1e-10 * kappa),
                      (rwsolve.MODE_DIRECT, 1e-8)):
        tau = np.empty_like(g)
        u = np.empty((nrhs, 2 * tg[0].size))
        info = r.solve(g, tau, nrhs=nrhs, targets=np.ascontiguousarray(np.stack(tg, 1)), u=u, mode=mode)
        err = (np.linalg.norm(tau - tau_or, axis=1) / nrm).max()
        res = (np.linalg.norm(A_or @ tau.T - g_or, axis=0) / np.linalg.norm(g_or, axis=0)).max()
        print(f"{kind} P={P} holes P={PH} mode={mode}: density error {err:.2e}, residual {res:.2e}, "
              f"cond(A_nn) {kappa:.1e}, iters {info['iters']}")
        assert err <= bar, (mode, err)
        if mode == rwsolve.MODE_GMRES_FP32:
            # FGMRES stops on the ELS residual; the exact operator differs from
            # the ELS one by the 1e-12 compression
            assert info["rel_residual"] <= 1e-10 and res <= 1e-9
        uu = u.reshape(nrhs, -1, 2).transpose(1, 2, 0)
        u_or = H.velocity(wall_o, hn, tau.T, *tg)
        assert np.abs(uu - u_or).max() <= 1e-12 * np.abs(u_or).max()
        assert np.abs(uu - ue).max() <= max(1e-10, 10 * bar) * np.abs(ue).max()
    # pressure of the refined-mode density: oracle evaluation and closed form
    tau = np.empty_like(g)
    r.solve(g, tau, nrhs=nrhs, mode=rwsolve.MODE_DIRECT_REFINED)
    p = r.pressure(tau, np.ascontiguousarray(np.stack(tg, 1)), np.empty((nrhs, tg[0].size)), nrhs=nrhs)  # (nrhs, nt)
    p_or = H.pressure(wall_o, hn, tau.T, *tg)                             # (nt, nrhs)
    assert np.abs(p.T - p_or).max() <= 1e-12 * np.abs(p_or).max()
    pe = S.stokeslet_pressure(*tg, *src)
    d = p.T - pe
    assert np.abs(d - d.mean(axis=0)).max() <= 1e-8 * np.abs(pe).max()
    r.close()
    w.close()


def test_channel1024_paper_holes_sampled_rows(lib):
    nrhs = 2
    w, wall_o, hl, src = _case("channel", 1024, 10, nrhs=nrhs)
    r = w.add_holes(hl)
    st = r.stats()
    print("channel1024 + 3 holes:", st)
    hn = H.hole_nodes(hl)
    g = _device_data(r, src, nrhs)
    tau = np.empty_like(g)
    r.solve(g, tau, nrhs=nrhs, mode=rwsolve.MODE_DIRECT_REFINED)
    g_or = H.boundary_data(wall_o, hn, *src)
    rows = inputs.rng(77).choice(g_or.shape[0], 32, replace=False)
    rows = np.concatenate([rows, g_or.shape[0] - 1 - inputs.rng(78).choice(2 * hn["x"].size, 8, replace=False)])
    res = H.apply_rows(wall_o, hn, hl, tau.T, rows) - g_or[rows]
    rel = np.abs(res).max() / np.abs(g_or).max()
    print(f"sampled residual / max|g| = {rel:.2e}")
    assert rel <= 1e-9
    tg = inputs.targets_fluid(4, hl, "channel", 16)
    u = H.velocity(wall_o, hn, tau.T, *tg)
    ue = S.stokeslet_velocity(*tg, *src)
    assert np.abs(u - ue).max() <= 1e-9 * np.abs(ue).max()
    r.close()
    w.close()


def test_batch_mixes_holes_and_refinements(lib):
    w, wall_o, hl, src = _case("star", 32, 6)
    r1 = w.add_holes(hl)
    r2 = w.refine([30, 31, 0], [2, 3, 2])
    b = rwsolve.Batch([r1, r2])
    nrhs = 2
    g1 = _device_data(r1, src, nrhs)
    sx, sy, f = inputs.stokeslets_star(5, nrhs=nrhs)
    g2 = _device_data(r2, (sx, sy, f), nrhs)
    gall = np.ascontiguousarray(np.concatenate([g1, g2], axis=1))
    out = np.empty_like(gall)
    b.solve(gall, out, nrhs=nrhs, use_graph=True)
    for r, g, (lo, hi) in ((r1, g1, (b.offsets[0], b.offsets[1])), (r2, g2, (b.offsets[1], b.offsets[2]))):
        t = np.empty_like(g)
        r.solve(g, t, nrhs=nrhs, mode=rwsolve.MODE_DIRECT)
        assert np.abs(out[:, lo:hi] - t).max() <= 1e-12 * np.abs(t).max()
    b.close()
    r1.close()
    r2.close()
    w.close()


@pytest.mark.parametrize("bad", [
    [dict(cx=0.3, cy=0.0, R=0.2, P=6), dict(cx=0.45, cy=0.0, R=0.2, P=6)],   # overlapping
    [dict(cx=0.3, cy=0.0, R=0.1, P=4)],                                       # too few panels
    [dict(cx=0.3, cy=0.0, R=-0.1, P=6)],                                      # negative radius
    [dict(cx=0.3, cy=0.0, R=0.1, a=1.2, k=3, P=6)],                           # self-intersecting shape
    [dict(cx=0.3, cy=0.0, R=0.1, P=70)],                                      # more than 1024 points
])
def test_invalid_holes_rejected(lib, bad):
    w = rwsolve.Wall("star", 16, (0.3, 5, 1.0))
    with pytest.raises(rwsolve.RWError) as e:
        w.add_holes(bad)
    assert e.value.code == -1
    w.close()
