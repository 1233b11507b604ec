"""Batched single-launch solve (rw_batch_*): the stacked solution of several
refinements on different walls equals each refinement's own rw_solve, with
and without CUDA-graph replay.  Tolerances: 1e-13 relative at the default
tile height (the same products in the same order); 1e-11 after the
autotuner picks another tile height (each row's dot products are summed in
another order: FP64 rounding, amplified by kappa(A) ~ 5e2)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import rwsolve, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_batch_equals_individual_solves():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rwsolve.load(build_if_missing=True)
    specs = [(0.3, 5, 64, [60, 61, 62, 63, 0], 2), (0.15, 3, 40, [7, 8], 3), (0.4, 8, 96, [50], 4)]
    walls, refs = [], []
    for a, k, P, panels, L in specs:
        w = rwsolve.Wall("star", P, (a, k, 1.0))
        walls.append(w)
        refs.append(w.refine(panels, [L] * len(panels)))
    nrhs = 3
    gs, taus = [], []
    for i, r in enumerate(refs):
        sx, sy, f = inputs.stokeslets_star(20 + i, nrhs=nrhs)
        g = np.empty((nrhs, 2 * r.stats()["n_n"]))
        r.stokeslet_data(np.stack([sx, sy], 1), np.transpose(f, (2, 0, 1)).copy(), g, nrhs=nrhs)
        t = np.empty_like(g)
        r.solve(g, t, nrhs=nrhs)
        gs.append(g)
        taus.append(t)
    b = rwsolve.Batch(refs)
    G = b.offsets[-1]
    gall = np.concatenate(gs, axis=1)             # (nrhs, G): column-major G x nrhs
    assert gall.shape == (nrhs, G)
    for use_graph in (False, True, True):
        out = np.full((nrhs, G), np.nan)
        b.solve(np.ascontiguousarray(gall), out, nrhs=nrhs, use_graph=use_graph)
        for i in range(len(refs)):
            assert rel(out[:, b.offsets[i]:b.offsets[i + 1]], taus[i]) < 1e-13
    tr, ms = b.autotune(nrhs=nrhs)
    assert tr in (16, 32, 64) and ms > 0
    out = np.empty((nrhs, G))
    b.solve(np.ascontiguousarray(gall), out, nrhs=nrhs, use_graph=True)
    for i in range(len(refs)):
        assert rel(out[:, b.offsets[i]:b.offsets[i + 1]], taus[i]) < (1e-13 if tr == 32 else 1e-11)
    b.close()
    for r in refs:
        r.close()
    for w in walls:
        w.close()
