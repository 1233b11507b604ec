"""Host-side checks that need no GPU: the C-ABI library builds, loads and
exports every function include/rwsolve.h declares; argument validation
rejects bad input before any device work; the seeded input generators are
deterministic."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2108_07205_gb300 import rwsolve, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "rwsolve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rw_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    L = rwsolve.load(build_if_missing=True)
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(rwsolve.EXPORTS)


def test_default_opts_and_validation_without_gpu():
    L = rwsolve.load(build_if_missing=True)
    o = rwsolve.default_opts()
    assert o.leaf_points == 64 and o.id_tol == 1e-12 and o.gmres_tol == 1e-10
    # the last field of rw_opts: a layout mismatch between the header and the
    # binding would leave it unset or shifted
    assert o.hole_div_ratio == 4.0 and o.seed == 0x5eed2108 and o.op_tol == 0.0
    bad_op = rwsolve.default_opts(op_tol=-1e-14)
    d1 = rwsolve.WallDesc()
    d1.curve_kind = rwsolve.CURVE_STAR
    d1.n_panels = 8
    h1 = ctypes.c_void_p()
    assert L.rw_hbs_build(ctypes.byref(d1), ctypes.byref(bad_op), None, ctypes.byref(h1)) == -1
    assert b"op_tol" in L.rw_last_error()
    bad_mf = rwsolve.default_opts(mixed_factor=3)
    assert L.rw_hbs_build(ctypes.byref(d1), ctypes.byref(bad_mf), None, ctypes.byref(h1)) == -1
    assert b"mixed_factor" in L.rw_last_error()
    bad = rwsolve.default_opts(hole_div_ratio=1.2)   # must exceed bas_ratio (1.5)
    d0 = rwsolve.WallDesc()
    d0.curve_kind = rwsolve.CURVE_STAR
    d0.n_panels = 8
    h0 = ctypes.c_void_p()
    assert L.rw_hbs_build(ctypes.byref(d0), ctypes.byref(bad), None, ctypes.byref(h0)) == -1
    assert b"hole_div_ratio" in L.rw_last_error()
    d = rwsolve.WallDesc()
    d.curve_kind = 7
    d.n_panels = 4
    h = ctypes.c_void_p()
    assert L.rw_hbs_build(ctypes.byref(d), None, None, ctypes.byref(h)) == -1
    assert b"curve" in L.rw_last_error()
    d.curve_kind = rwsolve.CURVE_STAR
    d.n_panels = 0
    assert L.rw_hbs_build(ctypes.byref(d), None, None, ctypes.byref(h)) == -1
    bad = rwsolve.default_opts(id_tol=2.0)
    d.n_panels = 8
    assert L.rw_hbs_build(ctypes.byref(d), ctypes.byref(bad), None, ctypes.byref(h)) == -1
    assert b"id_tol" in L.rw_last_error()
    assert L.rw_refine_factor(None, 1, None, None, None, ctypes.byref(h)) == -1
    assert L.rw_solve(None, 1, None, None, 0, None, None, 0, None, None) == -1
    with pytest.raises(TypeError):
        rwsolve._ptr(np.zeros(3, dtype=np.float32))


def test_exterior_build_validation_without_gpu():
    L = rwsolve.load(build_if_missing=True)
    h = ctypes.c_void_p()
    assert L.rw_hbs_build_exterior(None, None, None, ctypes.byref(h)) == -1
    d = rwsolve.WallDesc()
    d.curve_kind = rwsolve.CURVE_STAR
    d.n_panels = 4
    assert L.rw_hbs_build_exterior(ctypes.byref(d), None, None, ctypes.byref(h)) == -1
    assert b"at least 8 panels" in L.rw_last_error()
    d.curve_kind = 7
    d.n_panels = 64
    assert L.rw_hbs_build_exterior(ctypes.byref(d), None, None, ctypes.byref(h)) == -1
    assert b"unknown curve kind" in L.rw_last_error()


def test_nodes_and_checkpoint_validation_without_gpu(tmp_path):
    L = rwsolve.load(build_if_missing=True)
    h = ctypes.c_void_p()
    assert L.rw_hbs_build_nodes(None, None, None, ctypes.byref(h)) == -1
    nd = rwsolve.NodesDesc(5, None, None, None, None, None, None)
    assert L.rw_hbs_build_nodes(ctypes.byref(nd), None, None, ctypes.byref(h)) == -1
    assert b"multiple of 16" in L.rw_last_error()
    assert L.rw_refine_factor_nodes(None, 1, None, None, None, None, ctypes.byref(h)) == -1
    hole = rwsolve.HoleDesc(0.3, 0.0, 0.1, 0.0, 1, 10)
    assert L.rw_holes_factor(None, 1, ctypes.byref(hole), None, ctypes.byref(h)) == -1
    assert L.rw_holes_factor(None, 0, None, None, ctypes.byref(h)) == -1
    assert L.rw_hbs_load(os.fsencode(str(tmp_path / "missing.rw")), None, ctypes.byref(h)) == -1
    assert b"cannot open" in L.rw_last_error()
    junk = tmp_path / "junk.rw"
    junk.write_bytes(b"not a wall file at all")
    assert L.rw_hbs_load(os.fsencode(str(junk)), None, ctypes.byref(h)) == -1
    assert b"not a wall file" in L.rw_last_error()
    assert L.rw_hbs_save(None, b"x.rw") == -1


def test_inputs_are_seeded():
    a = inputs.refinement_window(3, 64, 4, 2, 5)
    b = inputs.refinement_window(3, 64, 4, 2, 5)
    assert a == b and len(a[0]) == 4 and all(2 <= L <= 5 for L in a[1])
    s1 = inputs.time_schedule(0, 1024, 5)
    assert [p[0][0] for p in s1] == [(s1[0][0][0] + i) % 1024 for i in range(5)]
    x1 = inputs.stokeslets_channel(4)
    x2 = inputs.stokeslets_channel(4)
    assert all(np.array_equal(u, v) for u, v in zip(x1, x2))
    assert np.all(np.abs(x1[1]) >= 1.0)
