"""The allocation-free inverse sweep (rw_hbs_apply_inverse_noalloc).

It exists for callers that cannot let the library allocate device memory
during a solve (their device memory belongs to another framework's pool, or
an allocation could stall a latency-critical loop).  Through the C ABI, its
output must match rw_hbs_apply_inverse within the tolerance of the other
sweep tests (1e-13 relative; the same kernels run in the same order, so the
results are expected to agree to rounding), on two calls in a row on the same
stream (the shared scratch array keeps the first call's contents).  This file
is collected last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_07205_gb300 import rwsolve, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_inverse_matches_regular_sweep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = rwsolve.load(build_if_missing=True)
    wall = rwsolve.Wall("star", 64, (0.3, 5, 1.0))
    n2 = 2 * wall.stats()["n_points"]
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    for call, nrhs in enumerate((3, 3)):
        b = torch.from_numpy(inputs.rng(10 + call).standard_normal((nrhs, n2))).cuda()
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
