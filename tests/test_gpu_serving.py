"""Serving loop (rw_server_*): continuous batching of refined-wall solve
requests over resident walls.  Each result must be the same alone and in the
mix (tolerance 1e-13 relative; the kernels are deterministic, so equality is
expected), must match the single-request API (rw_refine_factor + rw_solve),
and a budget too small for two requests must still serve them one at a time."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import rwsolve, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def forces(seed, nrhs):
    sx, sy, f = inputs.stokeslets_star(seed, nrhs=nrhs)
    return np.stack([sx, sy], 1), np.transpose(f, (2, 0, 1)).copy()


@pytest.fixture(scope="module")
def walls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rwsolve.load(build_if_missing=True)
    a = rwsolve.Wall("star", 64, (0.3, 5, 1.0))
    b = rwsolve.Wall("star", 48, (0.2, 3, 1.0))
    yield a, b
    a.close()
    b.close()


def test_alone_equals_in_the_mix(walls):
    a, b = walls
    tg = np.stack(inputs.targets_star(1, 8), 1)
    src, f = forces(0, 2)
    sv = rwsolve.Server(n_workers=4, max_device_bytes=32 << 30)
    t, tau_alone, u_alone = sv.submit(a, [10, 11, 12], [3, 3, 3], src, f, nrhs=2, targets=tg)
    sv.wait(t)
    # the same request among a dozen others of different walls, sizes and modes
    mix = []
    for i in range(12):
        w = a if i % 2 == 0 else b
        P = w.n_panels
        panels, levels = inputs.refinement_window(100 + i, P, 1 + i % 4, 1, 4)
        s2, f2 = forces(10 + i, 1 + i % 3)
        mode = rwsolve.MODE_GMRES_FP32 if i % 5 == 4 else rwsolve.MODE_DIRECT
        mix.append((w, panels, levels, s2, f2, 1 + i % 3, mode) + sv.submit(w, panels, levels, s2, f2, nrhs=1 + i % 3,
                                                                         mode=mode))
        if i == 5:
            t2, tau_mix, u_mix = sv.submit(a, [10, 11, 12], [3, 3, 3], src, f, nrhs=2, targets=tg)
    lat = [sv.wait(m[7]) for m in mix] + [sv.wait(t2)]
    assert all(x > 0 for x in lat)
    assert rel(tau_mix, tau_alone) < 1e-13 and rel(u_mix, u_alone) < 1e-13
    # each mixed result matches the single-request API
    for (w, panels, levels, s2, f2, nrhs, mode, _, tau, _) in mix[:6]:
        ref = w.refine(panels, levels)
        g = np.empty((nrhs, tau.shape[1]))
        ref.stokeslet_data(s2, f2, g, nrhs=nrhs)
        t_api = np.empty_like(g)
        ref.solve(g, t_api, nrhs=nrhs, mode=mode)
        assert rel(tau, t_api) < (1e-13 if mode == rwsolve.MODE_DIRECT else 1e-9)
        ref.close()
    sv.close()


def test_tiny_budget_serves_one_at_a_time(walls):
    a, _ = walls
    src, f = forces(3, 1)
    sv = rwsolve.Server(n_workers=3, max_device_bytes=1)
    tickets = [sv.submit(a, [p, p + 1], [2, 2], src, f)[0] for p in (4, 20, 40)]
    for t in tickets:
        sv.wait(t)
        assert sv.poll(t)[0] == 0
    sv.close()


def test_factor_cache_reuse(walls):
    """A repeated (wall, panels, levels) request reuses the cached factors:
    the same result as the first request, and a cache hit."""
    a, b = walls
    src, f = forces(3, 2)
    src2, f2 = forces(4, 2)
    sv = rwsolve.Server(n_workers=2, max_device_bytes=32 << 30, cache_bytes=8 << 30)
    t1, tau1, _ = sv.submit(a, [5, 6, 7], [2, 3, 2], src, f, nrhs=2)
    sv.wait(t1)
    t2, tau2, _ = sv.submit(a, [5, 6, 7], [2, 3, 2], src, f, nrhs=2)       # same key, same data
    t3, tau3, _ = sv.submit(a, [5, 6, 7], [2, 3, 2], src2, f2, nrhs=2)     # same key, new data
    t4, tau4, _ = sv.submit(b, [5, 6, 7], [2, 3, 2], src, f, nrhs=2)       # other wall: a miss
    for t in (t2, t3, t4):
        sv.wait(t)
    st = sv.stats()
    assert st["hits"] == 2 and st["misses"] == 2 and st["cache_bytes"] > 0
    assert np.array_equal(tau1, tau2)
    # the cached factors solve new data like a fresh factorisation
    r = a.refine([5, 6, 7], [2, 3, 2])
    g = np.empty((2, 2 * r.stats()["n_n"]))
    r.stokeslet_data(np.ascontiguousarray(src2), np.ascontiguousarray(f2), g, nrhs=2)
    tau_ref = np.empty_like(g)
    r.solve(g, tau_ref, nrhs=2)
    assert rel(tau3, tau_ref) <= 1e-13
    r.close()
    # disabling the cache frees it
    sv.set_cache(0)
    assert sv.stats()["cache_bytes"] == 0
    sv.close()
