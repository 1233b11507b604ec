"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (relative 2-norm unless stated), from the arithmetic:
* nodes, boundary data: 1e-13 (same formulas, different rounding order);
* HBS inverse vs dense solve: 1e-10 (compression tolerance 1e-12 times
  kappa(A_oo) ~ 3e2 on the star wall);
* refined density, RW_MODE_DIRECT_REFINED: 1e-10 (the parity bar for the
  FP64 path); RW_MODE_DIRECT alone: 1e-9 (1e-12 compression amplified by
  kappa(A_nn) ~ 5e2, measured 1.7e-10);
* mixed path (FP32 sweeps inside FP64 FGMRES): ELS residual <= 1e-10 and
  density within 1e-9 of the oracle (the ELS operator itself carries the
  1e-12 compression); the same with BF16 sweep matrices on the star wall,
  in more iterations than FP32;
* full-size channel (32768 unknowns): residual of the exact refined operator
  on 64 sampled rows computed one by one by the oracle, <= 1e-8 relative to
  max |g| (kappa(A) ~ 1e6 on this wall), and the interior velocity against the
  closed-form Stokeslet field <= 1e-8; the same bars on the 2048-panel
  channel (65536 unknowns) with 64 right-hand sides, direct and FGMRES.
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


@pytest.fixture(scope="module")
def star64(lib):
    w = rwsolve.Wall("star", 64, (0.3, 5, 1.0))
    yield w
    w.close()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def data(ref, o, seed, nrhs, kind="star"):
    if kind == "star":
        sx, sy, f = inputs.stokeslets_star(seed, nrhs=nrhs)
    else:
        sx, sy, f = inputs.stokeslets_channel(seed, nrhs=nrhs)
    src = np.ascontiguousarray(np.stack([sx, sy], 1))
    fd = np.ascontiguousarray(np.transpose(f, (2, 0, 1)))
    g = np.empty((nrhs, 2 * ref.stats()["n_n"]))
    ref.stokeslet_data(src, fd, g, nrhs=nrhs)
    g_or = None if o is None else S.boundary_data(o["n"], sx, sy, f).T
    return g, g_or, (sx, sy, f)


def test_wall_nodes(star64):
    nd = star64.nodes()
    on = D.wall_nodes("star", STAR, 64)
    for key in ("x", "y", "nx", "ny", "w", "kappa"):
        assert np.abs(nd[key] - on[key]).max() <= 1e-13 * (1 + np.abs(on[key]).max()), key


def test_hbs_inverse_and_forward_vs_dense(star64):
    on = D.wall_nodes("star", STAR, 64)
    A = S.matrix(on)
    b = inputs.rng(0).standard_normal((3, A.shape[0]))
    x = np.empty_like(b)
    star64.apply_inverse(b, x, nrhs=3)
    assert rel(x, np.linalg.solve(A, b.T).T) < 1e-10
    y = np.empty_like(b)
    star64.apply_forward(b, y, nrhs=3)
    assert rel(y, (A @ b.T).T) < 1e-11
    # many right-hand sides take the tiled GEMM path
    b12 = inputs.rng(1).standard_normal((12, A.shape[0]))
    x12 = np.empty_like(b12)
    star64.apply_inverse(b12, x12, nrhs=12)
    assert rel(x12, np.linalg.solve(A, b12.T).T) < 1e-10


def test_single_leaf_wall_is_dense_inverse(lib):
    w = rwsolve.Wall("star", 4, (0.2, 3, 1.0))
    assert w.stats()["levels"] == 0
    on = D.wall_nodes("star", dict(a=0.2, k=3), 4)
    A = S.matrix(on)
    b = inputs.rng(2).standard_normal(A.shape[0])
    x = np.empty_like(b)
    w.apply_inverse(b, x)
    assert rel(x, np.linalg.solve(A, b)) < 1e-13
    w.close()


@pytest.mark.parametrize("panels,levels", [
    (None, None),                          # seeded 4-panel window, 3 levels
    ([62, 63, 0, 1], [2, 3, 1, 2]),        # wrap-around window, ragged levels
    ([10], [2]),                           # 64 added points: dense A_pp
    ([30], [0]),                           # level 0: same points re-added
])
def test_refined_solve_vs_oracle(star64, panels, levels):
    if panels is None:
        panels, levels = inputs.refinement_window(0, 64, 4, 3, 3)
    ref = star64.refine(panels, levels)
    st = ref.stats()
    o = D.refine("star", STAR, 64, panels, levels)
    assert st["n_n"] == o["n"]["x"].size and st["n_p"] == o["p"]["x"].size
    rn = ref.nodes()
    for key in ("x", "y", "nx", "ny", "w", "kappa"):
        assert np.abs(rn[key] - o["n"][key]).max() <= 1e-13 * (1 + np.abs(o["n"][key]).max())
    g, g_or, (sx, sy, f) = data(ref, o, 0, 3)
    assert np.abs(g - g_or).max() <= 1e-13 * np.abs(g_or).max()
    tau_or = DN.solve_refined(o, g_or.T).T
    tau = np.empty_like(g)
    tx, ty = inputs.targets_star(1)
    tg = np.ascontiguousarray(np.stack([tx, ty], 1))
    u = np.empty((3, 2 * tx.size))
    ref.solve(g, tau, nrhs=3, targets=tg, u=u)
    assert rel(tau, tau_or) < 1e-9
    tau_r = np.empty_like(g)
    info = ref.solve(g, tau_r, nrhs=3, mode=rwsolve.MODE_DIRECT_REFINED)
    assert info["iters"] == 1
    assert rel(tau_r, tau_or) < 1e-10
    ue = np.transpose(S.stokeslet_velocity(tx, ty, sx, sy, f), (2, 0, 1)).reshape(3, -1)
    assert np.abs(u - ue).max() < 1e-9 * np.abs(ue).max()
    ref.close()


def test_mixed_gmres_fp32(star64):
    panels, levels = inputs.refinement_window(0, 64, 4, 3, 3)
    ref = star64.refine(panels, levels)
    o = D.refine("star", STAR, 64, panels, levels)
    g, g_or, _ = data(ref, o, 1, 4)
    tau = np.empty_like(g)
    info = ref.solve(g, tau, nrhs=4, mode=rwsolve.MODE_GMRES_FP32)
    assert info["rel_residual"] <= 1e-10
    assert 1 <= info["iters"] <= 10
    assert rel(tau, DN.solve_refined(o, g_or.T).T) < 1e-9
    ref.close()


def test_mixed_gmres_bf16(star64):
    # BF16 matrices in the preconditioner's sweeps (FP32 vectors and sums):
    # on this wall (kappa ~ 4e2) the preconditioned operator stays within
    # ~5e-2 of the identity, so FGMRES still reaches 1e-10, in more iterations
    panels, levels = inputs.refinement_window(0, 64, 4, 3, 3)
    ref = star64.refine(panels, levels)
    o = D.refine("star", STAR, 64, panels, levels)
    g, g_or, _ = data(ref, o, 1, 4)
    tau32, tau16 = np.empty_like(g), np.empty_like(g)
    i32 = ref.solve(g, tau32, nrhs=4, mode=rwsolve.MODE_GMRES_FP32)
    i16 = ref.solve(g, tau16, nrhs=4, mode=rwsolve.MODE_GMRES_BF16)
    assert i16["rel_residual"] <= 1e-10
    assert i32["iters"] < i16["iters"] <= 30
    assert rel(tau16, DN.solve_refined(o, g_or.T).T) < 1e-9
    ref.close()


def test_exact_operator_and_multi_rhs_consistency(star64):
    panels, levels = inputs.refinement_window(3, 64, 3, 2, 2)
    ref = star64.refine(panels, levels)
    o = D.refine("star", STAR, 64, panels, levels)
    A = S.matrix(o["n"])
    t = inputs.rng(3).standard_normal((2, A.shape[0]))
    y = np.empty_like(t)
    ref.apply_refined(t, y, nrhs=2)
    assert rel(y, (A @ t.T).T) < 1e-13
    g, _, _ = data(ref, None, 2, 3)
    tau3 = np.empty_like(g)
    ref.solve(g, tau3, nrhs=3)
    for r in range(3):
        t1 = np.empty((1, g.shape[1]))
        ref.solve(np.ascontiguousarray(g[r:r + 1]), t1)
        assert rel(t1[0], tau3[r]) < 1e-13
    # device buffers give the same answer as host buffers
    gd = torch.from_numpy(g).cuda()
    td = torch.empty_like(gd)
    ref.solve(gd, td, nrhs=3)
    torch.cuda.synchronize()
    assert rel(td.cpu().numpy(), tau3) < 1e-15
    ref.close()


def test_many_rhs_take_the_gemm_sweeps(star64):
    """From 16 right-hand sides the direct solve sweeps level by level with
    batched GEMMs instead of the GEMV program: same bar against the oracle,
    and the same solution as the program path (which sums in another order)."""
    panels, levels = inputs.refinement_window(0, 64, 4, 3, 3)
    ref = star64.refine(panels, levels)
    o = D.refine("star", STAR, 64, panels, levels)
    g, g_or, _ = data(ref, o, 11, 20)
    tau = np.empty_like(g)
    ref.solve(g, tau, nrhs=20)
    assert rel(tau, DN.solve_refined(o, g_or.T).T) < 1e-9
    tau8 = np.empty((8, g.shape[1]))
    ref.solve(np.ascontiguousarray(g[:8]), tau8, nrhs=8)
    assert rel(tau[:8], tau8) < 1e-11
    ref.close()


def test_invalid_refinements_rejected(star64):
    nine_regions = list(range(0, 18, 2))   # nine contiguous runs: more than the eight a refinement groups
    for panels, levels in ((nine_regions, [1] * 9), ([64], [1]), ([1, 2], [2, 13]), ([4, 4], [1, 1])):
        with pytest.raises(rwsolve.RWError) as e:
            star64.refine(panels, levels)
        assert e.value.code == -1


@pytest.mark.parametrize("level", [2, 5])
def test_channel_full_size(lib, level):
    w = rwsolve.Wall("channel", 1024)
    st = w.stats()
    assert st["n_points"] == 16384
    sched = inputs.time_schedule(0, 1024, 1, level_lo=level, level_hi=level)
    panels, levels = sched[0]
    ref = w.refine(panels, levels)
    s = ref.stats()
    o = D.refine("channel", {}, 1024, panels, levels)
    g, _, (sx, sy, f) = data(ref, None, 7, 1, kind="channel")
    tau = np.empty_like(g)
    tx, ty = inputs.targets_channel(3)
    tg = np.ascontiguousarray(np.stack([tx, ty], 1))
    u = np.empty((1, 2 * tx.size))
    ref.solve(g, tau, targets=tg, u=u)
    rows = inputs.rng(level).choice(2 * s["n_n"], 64, replace=False)
    gs = S.boundary_data(o["n"], sx, sy, f)[:, 0]
    assert np.abs(gs[rows] - g[0, rows]).max() <= 1e-13 * np.abs(gs).max()
    res = S.apply_rows(o["n"], tau[0], rows) - gs[rows]
    assert np.abs(res).max() <= 1e-8 * np.abs(gs).max()
    ue = S.stokeslet_velocity(tx, ty, sx, sy, f)[:, :, 0].reshape(-1)
    assert np.abs(u[0] - ue).max() <= 1e-8 * np.abs(ue).max()
    tau2 = np.empty_like(g)
    info = ref.solve(g, tau2, mode=rwsolve.MODE_GMRES_FP32)
    assert info["rel_residual"] <= 1e-10
    ref.close()
    w.close()


def test_mixed_config_full_size(lib):
    # the 2048-panel channel (65536 unknowns) with 64 right-hand sides, one
    # Stokeslet pair each, as the mixed-precision workload runs it: the direct
    # solve (level-by-level GEMM sweeps) and FP32-preconditioned FGMRES, both
    # checked on 24 rows of the exact refined operator written out by the
    # oracle, for every right-hand side, and on the closed-form velocity
    nrhs = 64
    w = rwsolve.Wall("channel", 2048)
    panels, levels = inputs.time_schedule(11, 2048, 1, level_lo=4, level_hi=4)[0]
    ref = w.refine(panels, levels)
    o = D.refine("channel", {}, 2048, panels, levels)
    sx, sy, f = inputs.stokeslet_pairs_channel(5, nrhs)
    g = np.empty((nrhs, 2 * ref.stats()["n_n"]))
    ref.stokeslet_data(np.ascontiguousarray(np.stack([sx, sy], 1)),
                       np.ascontiguousarray(np.transpose(f, (2, 0, 1))), g, nrhs=nrhs)
    rows = inputs.rng(21).choice(g.shape[1], 24, replace=False)
    # the oracle's data at the sampled rows only (every node x 128 sources x
    # 64 right-hand sides would not fit a test's memory)
    pts = rows // 2
    ur = S.stokeslet_velocity(o["n"]["x"][pts], o["n"]["y"][pts], sx, sy, f)   # (24, 2, nrhs)
    gr = ur[np.arange(rows.size), rows % 2, :]                                 # (24, nrhs)
    gmax = np.abs(g).max()
    assert np.abs(gr.T - g[:, rows]).max() <= 1e-13 * gmax
    tx, ty = inputs.targets_channel(4, 8)
    ue = S.stokeslet_velocity(tx, ty, sx, sy, f)                     # (nt, 2, nrhs)
    for mode in (rwsolve.MODE_DIRECT, rwsolve.MODE_GMRES_FP32):
        tau = np.empty_like(g)
        u = np.empty((nrhs, 2 * tx.size))
        info = ref.solve(g, tau, nrhs=nrhs, targets=np.ascontiguousarray(np.stack([tx, ty], 1)), u=u, mode=mode)
        res = S.apply_rows(o["n"], tau.T, rows) - gr
        assert np.abs(res).max() <= 1e-8 * gmax, mode
        uu = u.reshape(nrhs, -1, 2).transpose(1, 2, 0)
        assert np.abs(uu - ue).max() <= 1e-8 * np.abs(ue).max(), mode
        if mode == rwsolve.MODE_GMRES_FP32:
            assert info["rel_residual"] <= 1e-10
    ref.close()
    w.close()
