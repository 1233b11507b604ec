"""Batched single-launch solve (rw_batch_*): the stacked solution of several
refinements on different walls equals each refinement's own rw_solve, with
and without CUDA-graph replay; the batched iterative refinement certifies
every instance to 1e-10 against its exact refined operator.  Tolerances: 1e-13 relative at the default
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


def test_batch_iterative_refinement_certified():
    """rw_batch_solve_ir: the batch (a 256-panel and a 128-panel channel,
    kappa(A) ~ 1e6, and a star; one wall whose refinements compute X in
    double-FP32) is solved to a certified relative residual <= 1e-10 in
    batched launches (10 right-hand sides: two launches of 8 per program).
    Every instance's density meets 1e-10 against its exact refined operator
    (entries on the fly) and agrees with its own rw_solve in the same
    iterative mode to within what the conditioning allows; the direct batch
    solve refuses the factorisation whose X is not FP64."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rwsolve.load(build_if_missing=True)
    op = rwsolve.default_opts(op_tol=1e-14)
    opdf = rwsolve.default_opts(op_tol=1e-14, mixed_factor=2)
    walls = [rwsolve.Wall("channel", 256, opts=op), rwsolve.Wall("channel", 128, opts=opdf),
             rwsolve.Wall("star", 64, (0.3, 5, 1.0), opts=op)]
    wins = [inputs.refinement_window(31, 256, 8, 3, 3), inputs.refinement_window(32, 128, 6, 4, 4),
            ([60, 61, 62, 63, 0], [2] * 5)]
    refs = [w.refine(p, l) for w, (p, l) in zip(walls, wins)]
    modes = [rwsolve.MODE_DIRECT_IR, rwsolve.MODE_DIRECT_IR_DF, rwsolve.MODE_DIRECT_IR]
    nrhs = 10
    gs, taus = [], []
    for i, r in enumerate(refs):
        if i < 2:
            sx, sy, f = inputs.stokeslets_channel(40 + i, nrhs=nrhs)
        else:
            sx, sy, f = inputs.stokeslets_star(40 + i, nrhs=nrhs)
        g = np.empty((nrhs, 2 * r.stats()["n_n"]))
        r.stokeslet_data(np.ascontiguousarray(np.stack([sx, sy], 1)), np.transpose(f, (2, 0, 1)).copy(), g, nrhs=nrhs)
        t = np.empty_like(g)
        r.solve(g, t, nrhs=nrhs, mode=modes[i])
        gs.append(g)
        taus.append(t)
    b = rwsolve.Batch(refs)
    G = b.offsets[-1]
    gall = np.ascontiguousarray(np.concatenate(gs, axis=1))
    for _ in range(2):
        out = np.full((nrhs, G), np.nan)
        info = b.solve_ir(gall, out, nrhs=nrhs, tol=1e-10)
        assert info["rel_residual"] <= 1e-10
        for i, r in enumerate(refs):
            tau = np.ascontiguousarray(out[:, b.offsets[i]:b.offsets[i + 1]])
            y = np.empty_like(tau)
            r.apply_refined(tau, y, nrhs=nrhs)
            res = (np.linalg.norm(y - gs[i], axis=1) / np.linalg.norm(gs[i], axis=1)).max()
            d = (np.linalg.norm(tau - taus[i], axis=1) / np.linalg.norm(taus[i], axis=1)).max()
            print(f"batch IR instance {i}: corrections {info['iters']}, true residual {res:.2e}, vs own solve {d:.2e}")
            assert res <= 1e-10
            assert d <= 1e-7
    with pytest.raises(rwsolve.RWError) as e:
        b.solve(gall, np.empty((nrhs, G)), nrhs=nrhs)
    assert e.value.code == -1
    b.close()
    for r in refs:
        r.close()
    for w in walls:
        w.close()
