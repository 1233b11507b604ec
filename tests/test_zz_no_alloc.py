"""The allocation-free inverse sweep (rw_hbs_apply_inverse_noalloc).

It exists for callers that cannot let the library allocate device memory
during a solve (their device memory belongs to another framework's pool, or
an allocation could stall a latency-critical loop).  Through the C ABI, on two
calls in a row on the same stream (the shared scratch array keeps the first
call's contents), its output must match
  * rw_hbs_apply_inverse within the 1e-13 relative tolerance of the other
    sweep tests (for 1..8 right-hand sides that call runs the persistent solve
    program and this one runs per-level GEMV launches: the same FP64 products
    of the same factors, summed in a different order), and
  * the oracle's dense solve of A_oo on the same wall within the HBS
    inverse's accuracy (ID tolerance 1e-12 times the conditioning of A_oo).
A sweep too large for the scratch array is refused before anything is
launched: the output keeps its previous contents; one right-hand side on the
same large wall fits and agrees with the regular sweep to 1e-8 (a 327680-point
wall, whose conditioning magnifies the different summation orders).  This file is collected
last so that a run stopping at the first failure has already run every other
test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import rwsolve, inputs  # noqa: E402
from oracle import discretize as D, stokes as S  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_inverse_matches_regular_sweep_and_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = rwsolve.load(build_if_missing=True)
    wall = rwsolve.Wall("star", 64, (0.3, 5, 1.0))
    n2 = 2 * wall.stats()["n_points"]
    A = S.matrix(D.wall_nodes("star", dict(a=0.3, k=5), 64))
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    for call, nrhs in enumerate((3, 3)):
        bh = inputs.rng(10 + call).standard_normal((nrhs, n2))
        b = torch.from_numpy(bh).cuda()
        x_ref = torch.empty_like(b)
        x_new = torch.full_like(b, float("nan"))
        assert L.rw_hbs_apply_inverse(wall.h, nrhs, ctypes.c_void_p(b.data_ptr()),
                                      ctypes.c_void_p(x_ref.data_ptr()), sp) == 0
        rc = L.rw_hbs_apply_inverse_noalloc(wall.h, nrhs, ctypes.c_void_p(b.data_ptr()),
                                            ctypes.c_void_p(x_new.data_ptr()), sp)
        assert rc == 0, L.rw_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(x_new).all()
        assert rel(x_new, x_ref) < 1e-13
        x_or = np.linalg.solve(A, bh.T).T
        assert np.linalg.norm(x_new.cpu().numpy() - x_or) / np.linalg.norm(x_or) < 1e-9
    # sizes beyond the limit are rejected with a message, nothing launched
    b9 = torch.zeros((9, n2), dtype=torch.float64, device="cuda")
    x9 = torch.empty_like(b9)
    rc = L.rw_hbs_apply_inverse_noalloc(wall.h, 9, ctypes.c_void_p(b9.data_ptr()), ctypes.c_void_p(x9.data_ptr()), sp)
    assert rc == -1
    assert b"nrhs" in L.rw_last_error()
    # host buffers are refused (they would need a staging allocation)
    bh = np.zeros(n2)
    xh = np.zeros(n2)
    rc = L.rw_hbs_apply_inverse_noalloc(wall.h, 1, ctypes.c_void_p(bh.ctypes.data), ctypes.c_void_p(xh.ctypes.data), sp)
    assert rc == -1 and b"device memory" in L.rw_last_error()
    wall.close()


def test_noalloc_refuses_a_sweep_larger_than_the_array_before_launching():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = rwsolve.load(build_if_missing=True)
    # 20480 panels (327680 points): 8 right-hand sides need about 60 MB of
    # per-level vectors, more than the 32 MiB array
    wall = rwsolve.Wall("star", 20480, (0.3, 5, 1.0))
    n2 = 2 * wall.stats()["n_points"]
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    b = torch.ones((8, n2), dtype=torch.float64, device="cuda")
    x = torch.full_like(b, float("nan"))
    rc = L.rw_hbs_apply_inverse_noalloc(wall.h, 8, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), sp)
    assert rc == -1
    assert b"scratch" in L.rw_last_error()
    torch.cuda.synchronize()
    assert torch.isnan(x).all()
    # one right-hand side fits and matches the regular sweep; on this
    # 327680-point wall the two routes' different summation orders differ by
    # about 2e-9 relative (the inverse's entries grow with the wall's
    # conditioning), so the bar here is 1e-8
    x1 = torch.empty((1, n2), dtype=torch.float64, device="cuda")
    x1r = torch.empty_like(x1)
    assert L.rw_hbs_apply_inverse_noalloc(wall.h, 1, ctypes.c_void_p(b.data_ptr()),
                                          ctypes.c_void_p(x1.data_ptr()), sp) == 0, L.rw_last_error()
    assert L.rw_hbs_apply_inverse(wall.h, 1, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x1r.data_ptr()), sp) == 0
    torch.cuda.synchronize()
    assert rel(x1, x1r) < 1e-8
    wall.close()
