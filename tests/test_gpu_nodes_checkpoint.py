"""Walls given by explicit nodes, refinements with caller-supplied added nodes,
and checkpoint/restore of a built wall, through the C ABI.

* A wall built from the oracle's star nodes and refined with the oracle's added
  nodes must meet the FP64 parity bar against the oracle's dense LU solve
  (1e-10 with one refinement step), like the curve-built wall.
* A restored wall must give the same results as the one saved (same factors,
  same kernels: equal to rounding, 1e-14).
* rw_info reports the refinement's Woodbury size and a finite condition
  estimate of W >= 1.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import rwsolve, inputs  # noqa: E402
from oracle import discretize as D, stokes as S, dense as DN  # noqa: E402

pytestmark = pytest.mark.gpu

STAR = dict(a=0.3, k=5)
PANELS, LEVELS = [20, 21, 22], [2, 3, 2]


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return rwsolve.load(build_if_missing=True)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def solve(ref, seed=5, nrhs=2):
    sx, sy, f = inputs.stokeslets_star(seed, nrhs=nrhs)
    src = np.ascontiguousarray(np.stack([sx, sy], 1))
    fd = np.ascontiguousarray(np.transpose(f, (2, 0, 1)))
    g = np.empty((nrhs, 2 * ref.stats()["n_n"]))
    ref.stokeslet_data(src, fd, g, nrhs=nrhs)
    tau = np.empty_like(g)
    info = ref.solve(g, tau, nrhs=nrhs, mode=rwsolve.MODE_DIRECT_REFINED)
    return tau, info, (sx, sy, f)


def test_wall_from_nodes_and_added_nodes(lib):
    on = D.wall_nodes("star", STAR, 64)
    w = rwsolve.Wall.from_nodes(on)
    nd = w.nodes()
    for key in ("x", "y", "nx", "ny", "w", "kappa"):
        assert np.array_equal(nd[key], on[key]), key
    o = D.refine("star", STAR, 64, PANELS, LEVELS)
    with pytest.raises(rwsolve.RWError):
        w.refine(PANELS, LEVELS)  # a node wall has no curve to refine
    ref = w.refine(PANELS, LEVELS, added=o["p"])
    tau, info, (sx, sy, f) = solve(ref)
    tau_or = DN.solve_refined(o, S.boundary_data(o["n"], sx, sy, f)).T
    assert rel(tau, tau_or) < 1e-10
    st = ref.stats()
    assert info["k_woodbury"] == st["k"] > 0
    assert np.isfinite(info["cond_w"]) and info["cond_w"] >= 1.0
    # the same added nodes on a curve-built wall give the same solution
    wc = rwsolve.Wall("star", 64, (0.3, 5, 1.0))
    rc = wc.refine(PANELS, LEVELS, added=o["p"])
    tau_c, _, _ = solve(rc)
    assert rel(tau_c, tau) < 1e-11
    for h in (rc, wc, ref, w):
        h.close()


def test_added_nodes_checked(lib):
    w = rwsolve.Wall("star", 64, (0.3, 5, 1.0))
    o = D.refine("star", STAR, 64, PANELS, LEVELS)
    short = {k: v[:-16] for k, v in o["p"].items()}
    with pytest.raises(rwsolve.RWError):
        w.refine(PANELS, LEVELS, added=short)
    bad = {k: v.copy() for k, v in o["p"].items()}
    bad["nx"][3] *= 2.0
    with pytest.raises(rwsolve.RWError):
        w.refine(PANELS, LEVELS, added=bad)
    w.close()


def test_checkpoint_restore(lib, tmp_path):
    w = rwsolve.Wall("star", 64, (0.3, 5, 1.0))
    path = tmp_path / "star64.rw"
    w.save(path)
    w2 = rwsolve.Wall.load(path)
    assert w2.stats() == w.stats()
    b = inputs.rng(3).standard_normal((2, 2 * w.stats()["n_points"]))
    x1, x2 = np.empty_like(b), np.empty_like(b)
    w.apply_inverse(b, x1, nrhs=2)
    w2.apply_inverse(b, x2, nrhs=2)
    assert rel(x2, x1) < 1e-14
    t1, _, _ = solve(w.refine(PANELS, LEVELS))
    t2, _, _ = solve(w2.refine(PANELS, LEVELS))
    assert rel(t2, t1) < 1e-14
    # a truncated file is refused
    data = path.read_bytes()
    cut = tmp_path / "cut.rw"
    cut.write_bytes(data[: len(data) // 2])
    with pytest.raises(rwsolve.RWError):
        rwsolve.Wall.load(cut)
    w2.close()
    w.close()
