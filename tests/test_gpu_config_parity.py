"""Oracle parity on seeded samples of the batched and serving workloads.

Both workloads run on walls too large for a dense oracle solve, so each result
is checked against the definition on sampled rows:
- 32 residual rows of the exact refined operator A_nn per wall, each written
  out one at a time by the oracle, at <= 1e-9 of max |g|;
- the interior velocity against the closed-form Stokeslet field, where the
  targets are known to lie inside.

Batched: uneven star walls r = 1 + a cos(k t), a ~ U[0.1, 0.4], k ~ U{3..8},
P ~ U{128..1024}, each refined at a seeded window of U{2..16} panels by
U{2..4} levels, 8 right-hand sides, solved together by one persistent launch.

Serving: requests on resident walls (channel 512 panels, star 256 panels),
each refining U{1..64} panels by U{2..6} levels with U{1..8} right-hand sides,
the three solve modes mixed.  Bars per mode:
- RW_MODE_DIRECT_REFINED corrects against the exact operator: <= 1e-9 of
  max |g|.
- RW_MODE_DIRECT and FP32-preconditioned FGMRES both solve the compressed
  system (1e-12 IDs): their exact-operator residual is the compression error
  amplified by the conditioning of these strongly graded refinements (up to 64
  sub-panels beside a coarse panel), <= 1e-7 of max |g|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import rwsolve, inputs  # noqa: E402
from oracle import discretize as D, stokes as S  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return rwsolve.load(build_if_missing=True)


def check_rows(nodes, tau, g_or, seed, n_rows=32, bar=1e-9):
    """Residual of the exact operator on sampled rows (all right-hand sides),
    relative to max |g|; asserts the bar and returns the value."""
    rows = inputs.rng(seed).choice(g_or.shape[0], n_rows, replace=False)
    res = S.apply_rows(nodes, tau.T, rows) - g_or[rows]
    rel = np.abs(res).max() / np.abs(g_or).max()
    assert rel <= bar, rel
    return rel


def test_batched_uneven_walls_sample(lib):
    g0 = inputs.rng(555)
    nrhs = 8
    walls, refs, olds, data = [], [], [], []
    for i in range(6):
        a = float(g0.uniform(0.1, 0.4))
        k = int(g0.integers(3, 9))
        P = int(g0.integers(128, 1025))
        m = int(g0.integers(2, 17))
        L = int(g0.integers(2, 5))
        panels, levels = inputs.refinement_window(1000 + i, P, m, L, L)
        w = rwsolve.Wall("star", P, (a, k, 1.0))
        r = w.refine(panels, levels)
        sx, sy, f = inputs.stokeslets_star(2000 + i, nrhs=nrhs, radius=2.5)
        g = np.empty((nrhs, 2 * r.stats()["n_n"]))
        r.stokeslet_data(np.stack([sx, sy], 1), np.transpose(f, (2, 0, 1)).copy(), g, nrhs=nrhs)
        walls.append(w)
        refs.append(r)
        olds.append(D.refine("star", dict(a=a, k=k), P, panels, levels))
        data.append((g, sx, sy, f))
    b = rwsolve.Batch(refs)
    gall = np.ascontiguousarray(np.concatenate([d[0] for d in data], axis=1))
    out = np.empty_like(gall)
    b.solve(gall, out, nrhs=nrhs, use_graph=True)
    tx, ty = inputs.targets_star(9, 12)
    for i, (o, (g, sx, sy, f)) in enumerate(zip(olds, data)):
        tau = out[:, b.offsets[i]:b.offsets[i + 1]]
        g_or = S.boundary_data(o["n"], sx, sy, f)
        assert np.abs(g_or.T - g).max() <= 1e-13 * np.abs(g_or).max()
        check_rows(o["n"], tau, g_or, 30 + i)
        u = S.velocity(o["n"], tau.T, tx, ty)
        ue = S.stokeslet_velocity(tx, ty, sx, sy, f)
        assert np.abs(u - ue).max() <= 1e-8 * np.abs(ue).max()
    b.close()
    for h in refs + walls:
        h.close()


def test_serving_requests_sample(lib):
    chan = rwsolve.Wall("channel", 512)
    star = rwsolve.Wall("star", 256, (0.3, 5, 1.0))
    sv = rwsolve.Server(n_workers=3, max_device_bytes=64 << 30)
    reqs = []
    for i in range(8):
        g = inputs.rng(7000 + i)
        use_star = bool(g.integers(0, 2))
        w = star if use_star else chan
        P = 256 if use_star else 512
        m = int(g.integers(1, 65))
        L = int(g.integers(2, 7))
        nrhs = int(g.integers(1, 9))
        mode = (rwsolve.MODE_DIRECT, rwsolve.MODE_DIRECT_REFINED, rwsolve.MODE_GMRES_FP32)[i % 3]
        panels, _ = inputs.refinement_window(7000 + i, P, m, L, L)
        if use_star:
            sx, sy, f = inputs.stokeslets_star(7000 + i, nrhs=nrhs)
            tx, ty = inputs.targets_star(7000 + i, 8)
        else:
            sx, sy, f = inputs.stokeslets_channel(7000 + i, nrhs=nrhs)
            tx, ty = inputs.targets_channel(7000 + i, 8)
        tg = np.stack([tx, ty], 1)
        t, tau, u = sv.submit(w, panels, [L] * m, np.stack([sx, sy], 1), np.transpose(f, (2, 0, 1)).copy(),
                              nrhs=nrhs, targets=tg, mode=mode)
        reqs.append((t, tau, u, "star" if use_star else "channel", P, panels, [L] * m, sx, sy, f, tx, ty, mode))
    for i, (t, tau, u, kind, P, panels, levels, sx, sy, f, tx, ty, mode) in enumerate(reqs):
        sv.wait(t)
        o = D.refine(kind, dict(a=0.3, k=5) if kind == "star" else {}, P, panels, levels)
        g_or = S.boundary_data(o["n"], sx, sy, f)
        bar = 1e-9 if mode == rwsolve.MODE_DIRECT_REFINED else 1e-7
        rel = check_rows(o["n"], tau, g_or, 80 + i, bar=bar)
        print(f"request {i}: {kind} P={P} m={len(panels)} L={levels[0]} mode={mode} residual/max|g| = {rel:.2e}")
        ue = S.stokeslet_velocity(tx, ty, sx, sy, f)                 # (nt, 2, nrhs)
        uu = u.reshape(u.shape[0], -1, 2).transpose(1, 2, 0)         # (nt, 2, nrhs)
        assert np.abs(uu - ue).max() <= 1e-8 * np.abs(ue).max()
    sv.close()
    star.close()
    chan.close()
