"""rw_hbs_load refuses damaged wall files before anything reaches the device.

A minimal wall file is written here, field by field, in the library's
checkpoint layout (tag, curve, options, nodes, the HBS tree and its factors,
the operator flag, trailer): a 2-panel star whose HBS is one dense leaf.  The
intact file passes every check, so on a machine without a GPU its load gets
as far as the first device allocation (an RW_ERR_OOM or RW_ERR_CUDA failure,
never RW_ERR_INVALID); with a GPU it loads.  Each damaged copy (one offset
past its buffer, a node range that does not cover the wall, a truncated file,
an operator flag that contradicts the options, options rw_hbs_build would
refuse) must be refused with RW_ERR_INVALID and a message naming the damage.
No GPU is needed: the checks run on the host before the upload."""
import ctypes
import os
import struct

import numpy as np

from paper_2108_07205_gb300 import rwsolve

TAG = b"RWHBSv04"


class InternalOpts(ctypes.Structure):
    """The library's internal option record as the file stores it."""
    _fields_ = [("leaf_points", ctypes.c_int), ("id_tol", ctypes.c_double), ("n_proxy", ctypes.c_int),
                ("proxy_ratio", ctypes.c_double), ("n_proxy_refine", ctypes.c_int), ("div_ratio", ctypes.c_double),
                ("bas_ratio", ctypes.c_double), ("dense_pp_max_points", ctypes.c_int), ("sketch_cols", ctypes.c_int),
                ("sketch_width", ctypes.c_int), ("gmres_tol", ctypes.c_double), ("gmres_maxit", ctypes.c_int),
                ("gmres_restarts", ctypes.c_int), ("seed", ctypes.c_ulonglong), ("hole_div_ratio", ctypes.c_double),
                ("op_tol", ctypes.c_double), ("mixed_factor", ctypes.c_int)]


def default_internal_opts():
    o = InternalOpts()
    o.leaf_points, o.id_tol, o.n_proxy, o.proxy_ratio = 64, 1e-12, 64, 2.0
    o.n_proxy_refine, o.div_ratio, o.bas_ratio = 96, 2.0, 1.5
    o.dense_pp_max_points, o.sketch_cols, o.sketch_width = 64, 2048, 192
    o.gmres_tol, o.gmres_maxit, o.gmres_restarts = 1e-10, 30, 4
    o.seed, o.hole_div_ratio, o.op_tol, o.mixed_factor = 0x5eed2108, 4.0, 0.0, 0
    return o


def vec(fmt, values):
    values = list(values)
    return struct.pack("<q", len(values)) + struct.pack("<%d%s" % (len(values), fmt), *values)


def wall_file(opts=None, oD=0, root_hi=32, op_flag=0, truncate=False):
    """Bytes of a 2-panel star wall (N = 32 points, one dense 64 x 64 leaf)."""
    n = 32
    o = opts or default_internal_opts()
    t = np.linspace(0, 2 * np.pi, n, endpoint=False)
    nodes = np.concatenate([np.cos(t), np.sin(t), np.cos(t), np.sin(t), np.full(n, 2 * np.pi / n), np.ones(n)])
    b = bytearray(TAG)
    b += struct.pack("<i", rwsolve.CURVE_STAR) + struct.pack("<8d", 0.3, 5, 1, 0, 0, 0, 0, 0) + struct.pack("<i", 2)
    b += bytes(o)
    b += struct.pack("<i", n) + vec("d", nodes)
    # HBS: N, L, node count, nodes (lo, hi, k, m, skeleton rows, skeleton columns)
    b += struct.pack("<iiq", n, 0, 2)
    for lo, hi in ((0, 0), (0, root_hi)):
        b += struct.pack("<iiii", lo, hi, 0, 0) + vec("i", []) + vec("i", [])
    b += struct.pack("<q", 1)
    dense = np.eye(2 * n).ravel()
    for buf in ([], [], [], [], dense, [], dense):            # U, V*, E, F*, G, B, D
        b += vec("d", buf)
    for off in ([], [], [], [], [0], [], [], [oD]):           # oU, oV*, oE, oF*, oG, oB12, oB21, oD
        b += vec("Q", off)
    b += vec("i", [])                                          # rank offsets (none at the root)
    b += struct.pack("<i", op_flag)
    if not truncate:
        b += TAG
    return bytes(b)


def load(tmp_path, data, name):
    L = rwsolve.load(build_if_missing=True)
    p = tmp_path / name
    p.write_bytes(data)
    h = ctypes.c_void_p()
    rc = L.rw_hbs_load(os.fsencode(str(p)), None, ctypes.byref(h))
    msg = L.rw_last_error()
    if rc == 0:
        L.rw_hbs_free(h)
    return rc, msg


def test_internal_option_record_size():
    assert ctypes.sizeof(InternalOpts) == 120


def test_intact_file_passes_the_checks(tmp_path):
    rc, msg = load(tmp_path, wall_file(), "ok.rw")
    assert rc != -1, msg
    assert b"corrupt" not in msg and b"truncated" not in msg


def test_damaged_files_are_refused(tmp_path):
    bad_opts = default_internal_opts()
    bad_opts.leaf_points = 0
    cases = {
        "leaf D offset": wall_file(oD=1),
        "root range": wall_file(root_hi=31),
        "truncated": wall_file(truncate=True),
        "operator flag": wall_file(op_flag=1),
        "options": wall_file(opts=bad_opts),
    }
    for what, data in cases.items():
        rc, msg = load(tmp_path, data, what.replace(" ", "_") + ".rw")
        assert rc == -1, (what, rc, msg)
        assert what.encode() in msg, (what, msg)
