"""Pressure at interior targets (Sec. 2) through the C ABI.

* On the same density, the CUDA pressure equals the oracle's double-layer
  pressure sum to 1e-13 (same formula, different summation order).
* From the refined solve of Stokeslet data, the pressure equals the
  Stokeslet pressure up to one constant (the velocity fixes the pressure up to
  a constant): the spread of the difference is <= 1e-9 of the pressure's
  spread, the density's own accuracy bar.
* Host and device buffers give the same result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import rwsolve, inputs  # noqa: E402
from oracle import stokes as S  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return rwsolve.load(build_if_missing=True)


def test_pressure_vs_oracle_and_closed_form(lib):
    w = rwsolve.Wall("star", 64, (0.3, 5, 1.0))
    ref = w.refine([62, 63, 0, 1], [3, 3, 2, 3])
    sx, sy, f = inputs.stokeslets_star(0, nrhs=2)
    src = np.ascontiguousarray(np.stack([sx, sy], 1))
    fd = np.ascontiguousarray(np.transpose(f, (2, 0, 1)))
    g = np.empty((2, 2 * ref.stats()["n_n"]))
    ref.stokeslet_data(src, fd, g, nrhs=2)
    tau = np.empty_like(g)
    ref.solve(g, tau, nrhs=2, mode=rwsolve.MODE_DIRECT_REFINED)
    tx, ty = inputs.targets_star(1, 24)
    tg = np.ascontiguousarray(np.stack([tx, ty], 1))
    p = np.empty((2, tx.size))
    ref.pressure(tau, tg, p, nrhs=2)
    p_or = S.pressure(ref.nodes(), tau.T, tx, ty).T
    assert np.abs(p - p_or).max() <= 1e-13 * np.abs(p_or).max()
    pe = S.stokeslet_pressure(tx, ty, sx, sy, f).T
    dif = p - pe
    spread = np.abs(dif - dif.mean(axis=1, keepdims=True)).max()
    assert spread <= 1e-9 * np.abs(pe - pe.mean(axis=1, keepdims=True)).max()
    # device buffers
    dev = torch.device("cuda")
    pd = torch.empty((2, tx.size), dtype=torch.float64, device=dev)
    ref.pressure(torch.from_numpy(tau).to(dev), torch.from_numpy(tg).to(dev), pd, nrhs=2)
    torch.cuda.synchronize()
    assert np.array_equal(pd.cpu().numpy(), p)
    ref.close()
    w.close()
