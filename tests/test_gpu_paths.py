"""Alternative kernel routes against the oracle.

The tuning switches change only how the same factorisations are scheduled:
- the cluster-only QR instead of the grid-wide one;
- other Gauss-Jordan cluster sizes and smallest QR clusters;
- a deep binary far-field tree (64-row chunks, pairwise merges to the top);
- no L2 prefetch in the solve program;
- no recompression (the blockwise ranks kept).

Each configuration must still meet the FP64 parity bar against the oracle's
dense LU solve of the refined system: 1e-10 relative with one refinement
step, the same bar as `test_gpu_parity`. Every configuration runs in a child
process, because the switches are read once per process.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import inputs  # noqa: E402
from oracle import discretize as D, stokes as S, dense as DN  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STAR = dict(a=0.3, k=5)
PANELS, LEVELS = [62, 63, 0, 1, 2, 3], [3, 4, 2, 3, 1, 2]

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2108_07205_gb300 import rwsolve, inputs
rwsolve.load(build_if_missing=False)
w = rwsolve.Wall("star", 64, (0.3, 5, 1.0))
r = w.refine([62, 63, 0, 1, 2, 3], [3, 4, 2, 3, 1, 2])
sx, sy, f = inputs.stokeslets_star(7, nrhs=2)
src = np.ascontiguousarray(np.stack([sx, sy], 1))
fd = np.ascontiguousarray(np.transpose(f, (2, 0, 1)))
g = np.empty((2, 2 * r.stats()["n_n"]))
r.stokeslet_data(src, fd, g, nrhs=2)
tau = np.empty_like(g)
r.solve(g, tau, nrhs=2, mode=rwsolve.MODE_DIRECT_REFINED)
np.save(sys.argv[2], tau)
r.close()
w.close()
"""


@pytest.fixture(scope="module")
def tau_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_07205_gb300 import rwsolve
    rwsolve.load(build_if_missing=True)
    o = D.refine("star", STAR, 64, PANELS, LEVELS)
    sx, sy, f = inputs.stokeslets_star(7, nrhs=2)
    g_or = S.boundary_data(o["n"], sx, sy, f)
    return DN.solve_refined(o, g_or).T


@pytest.mark.parametrize("env", [
    {},
    {"RW_ID_GRID": "0"},
    {"RW_GJ_CS": "1"},
    {"RW_GJ_CS": "4"},
    {"RW_ID_CS_MIN": "8"},
    {"RW_TREE_CHUNK": "64", "RW_ROOT_MERGE": "2"},
    {"RW_PROG_PREFETCH": "0"},
    {"RW_RECOMPRESS": "0"},
], ids=lambda e: ",".join(f"{k}={v}" for k, v in e.items()) or "default")
def test_route_matches_oracle(tau_oracle, env, tmp_path):
    out = tmp_path / "tau.npy"
    full = dict(os.environ)
    full.update(env)
    res = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(out)], env=full, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    tau = np.load(out)
    err = np.linalg.norm(tau - tau_oracle) / np.linalg.norm(tau_oracle)
    assert err < 1e-10, err
