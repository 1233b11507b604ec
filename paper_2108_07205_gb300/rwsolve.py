"""Thin Python binding of the rwsolve C ABI (include/rwsolve.h).

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/librwsolve.so``.  Arrays may be numpy arrays (host memory) or torch
CUDA tensors (device memory); FP64, column-major as the header states (a
C-contiguous numpy array of shape (nrhs, 2N) is the column-major 2N x nrhs
matrix).  Streams are torch.cuda streams or raw cudaStream_t integers.

Loading fails loudly if the library is missing: there is no fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

RW_OK = 0
ERRORS = {-1: "RW_ERR_INVALID", -2: "RW_ERR_OOM", -3: "RW_ERR_SINGULAR",
          -4: "RW_ERR_NOT_CONVERGED", -5: "RW_ERR_TIMEOUT", -6: "RW_ERR_CUDA"}
CURVE_STAR, CURVE_CHANNEL, CURVE_NODES = 0, 1, 2
MODE_DIRECT, MODE_GMRES_FP32, MODE_DIRECT_REFINED, MODE_GMRES_BF16 = 0, 1, 2, 3
MODE_DIRECT_IR, MODE_GMRES_MIXED, MODE_DIRECT_IR_DF = 4, 5, 6


class RWError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class WallDesc(ctypes.Structure):
    _fields_ = [("curve_kind", ctypes.c_int), ("n_panels", ctypes.c_int), ("params", ctypes.c_double * 8)]


class Opts(ctypes.Structure):
    _fields_ = [("leaf_points", ctypes.c_int), ("id_tol", ctypes.c_double), ("n_proxy", ctypes.c_int),
                ("proxy_ratio", ctypes.c_double), ("n_proxy_refine", ctypes.c_int),
                ("div_ratio", ctypes.c_double), ("bas_ratio", ctypes.c_double),
                ("dense_pp_max_points", ctypes.c_int), ("sketch_cols", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("gmres_maxit", ctypes.c_int),
                ("gmres_restarts", ctypes.c_int), ("seed", ctypes.c_ulonglong), ("hole_div_ratio", ctypes.c_double),
                ("op_tol", ctypes.c_double), ("mixed_factor", ctypes.c_int)]


class HbsStats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int), ("levels", ctypes.c_int), ("max_rank", ctypes.c_int),
                ("inv_elems", ctypes.c_longlong), ("fwd_elems", ctypes.c_longlong), ("bytes", ctypes.c_longlong),
                ("op_fwd_elems", ctypes.c_longlong)]


class RefStats(ctypes.Structure):
    _fields_ = [("n_k", ctypes.c_int), ("n_c", ctypes.c_int), ("n_p", ctypes.c_int), ("n_n", ctypes.c_int),
                ("n_ext", ctypes.c_int), ("k_far", ctypes.c_int), ("k_near", ctypes.c_int),
                ("k_pk", ctypes.c_int), ("k", ctypes.c_int), ("pp_dense", ctypes.c_int),
                ("pp_levels", ctypes.c_int), ("bytes", ctypes.c_longlong)]


class KernelStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


KCLASSES = ["id", "gemm", "gemv", "inverse", "eval", "other", "gemm_f32", "gemm_df"]


class Request(ctypes.Structure):
    _fields_ = [("wall", ctypes.c_void_p), ("n_cut", ctypes.c_int), ("panel_ids", ctypes.POINTER(ctypes.c_int)),
                ("levels", ctypes.POINTER(ctypes.c_int)), ("nrhs", ctypes.c_int), ("n_src", ctypes.c_int),
                ("src", ctypes.c_void_p), ("f", ctypes.c_void_p), ("n_targets", ctypes.c_int),
                ("targets", ctypes.c_void_p), ("tau", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("mode", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_residual", ctypes.c_double), ("k_woodbury", ctypes.c_int),
                ("cond_w", ctypes.c_double)]


class HoleDesc(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("radius", ctypes.c_double), ("a", ctypes.c_double),
                ("k", ctypes.c_int), ("n_panels", ctypes.c_int)]


class NodesDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("nx", ctypes.c_void_p),
                ("ny", ctypes.c_void_p), ("w", ctypes.c_void_p), ("kappa", ctypes.c_void_p)]


EXPORTS = ["rw_default_opts", "rw_hbs_build", "rw_hbs_build_exterior", "rw_hbs_build_nodes", "rw_hbs_save", "rw_hbs_load",
           "rw_refine_factor_nodes", "rw_holes_factor",
           "rw_hbs_stats_get", "rw_hbs_nodes", "rw_hbs_apply_inverse",
           "rw_hbs_apply_inverse_noalloc",
           "rw_hbs_apply_forward", "rw_refine_factor", "rw_ref_stats_get", "rw_ref_nodes", "rw_apply_refined",
           "rw_stokeslet_data", "rw_pressure",
           "rw_solve", "rw_batch_create", "rw_batch_rows", "rw_batch_autotune", "rw_batch_solve", "rw_batch_solve_ir",
           "rw_batch_free", "rw_server_create", "rw_server_submit", "rw_server_poll", "rw_server_wait",
           "rw_server_destroy", "rw_server_set_cache", "rw_server_stats", "rw_kernel_launches", "rw_profile", "rw_profile_read", "rw_ref_free", "rw_hbs_free", "rw_last_error"]

_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load librwsolve.so (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"rwsolve CUDA library not built: {path} missing (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p
    L.rw_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.rw_hbs_build.argtypes = [ctypes.POINTER(WallDesc), ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    L.rw_hbs_build_exterior.argtypes = [ctypes.POINTER(WallDesc), ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    L.rw_hbs_stats_get.argtypes = [vp, ctypes.POINTER(HbsStats)]
    L.rw_hbs_nodes.argtypes = [vp, dp, vp]
    L.rw_hbs_apply_inverse.argtypes = [vp, ctypes.c_int, dp, dp, vp]
    L.rw_hbs_apply_forward.argtypes = [vp, ctypes.c_int, dp, dp, vp]
    L.rw_hbs_apply_inverse_noalloc.argtypes = [vp, ctypes.c_int, dp, dp, vp]
    L.rw_refine_factor.argtypes = [vp, ctypes.c_int, ip, ip, vp, ctypes.POINTER(vp)]
    L.rw_hbs_build_nodes.argtypes = [ctypes.POINTER(NodesDesc), ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    L.rw_refine_factor_nodes.argtypes = [vp, ctypes.c_int, ip, ip, ctypes.POINTER(NodesDesc), vp, ctypes.POINTER(vp)]
    L.rw_holes_factor.argtypes = [vp, ctypes.c_int, ctypes.POINTER(HoleDesc), vp, ctypes.POINTER(vp)]
    L.rw_hbs_save.argtypes = [vp, ctypes.c_char_p]
    L.rw_hbs_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
    L.rw_ref_stats_get.argtypes = [vp, ctypes.POINTER(RefStats)]
    L.rw_ref_nodes.argtypes = [vp, dp, vp]
    L.rw_apply_refined.argtypes = [vp, ctypes.c_int, dp, dp, vp]
    L.rw_stokeslet_data.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int, dp, dp, vp]
    L.rw_pressure.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int, dp, dp, vp]
    L.rw_solve.argtypes = [vp, ctypes.c_int, dp, dp, ctypes.c_int, dp, dp, ctypes.c_int, vp, ctypes.POINTER(Info)]
    L.rw_ref_free.argtypes = [vp]
    L.rw_hbs_free.argtypes = [vp]
    L.rw_last_error.restype = ctypes.c_char_p
    L.rw_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp), vp, ctypes.POINTER(vp)]
    L.rw_batch_rows.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.rw_batch_autotune.argtypes = [vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
    L.rw_batch_solve.argtypes = [vp, ctypes.c_int, dp, dp, ctypes.c_int, vp]
    L.rw_batch_solve_ir.argtypes = [vp, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int, vp,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.rw_batch_free.argtypes = [vp]
    L.rw_server_create.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(vp)]
    L.rw_server_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_longlong)]
    L.rw_server_poll.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.rw_server_wait.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double)]
    L.rw_server_destroy.argtypes = [vp]
    L.rw_server_set_cache.argtypes = [vp, ctypes.c_longlong]
    L.rw_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                  ctypes.POINTER(ctypes.c_longlong)]
    L.rw_profile.argtypes = [ctypes.c_int]
    L.rw_profile_read.argtypes = [ctypes.POINTER(KernelStat), ctypes.c_int]
    L.rw_kernel_launches.argtypes = []
    L.rw_kernel_launches.restype = ctypes.c_ulonglong
    for name in EXPORTS:
        if name not in ("rw_last_error", "rw_ref_free", "rw_hbs_free", "rw_kernel_launches", "rw_batch_free"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc):
    if rc != RW_OK:
        raise RWError(rc, load().rw_last_error().decode())


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(a, writable=False):
    """Raw pointer of a numpy FP64 C-contiguous array or a torch FP64 tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("torch tensors must be contiguous float64")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("numpy arrays must be C-contiguous float64")
    if writable and not a.flags["WRITEABLE"]:
        raise TypeError("output array is read-only")
    return ctypes.c_void_p(a.ctypes.data)


def kernel_launches():
    """Kernels launched by the library so far in this process."""
    return int(load().rw_kernel_launches())


def profile(enable):
    """Start (True, clearing old records) or stop the kernel profiler."""
    _check(load().rw_profile(1 if enable else 0))


def profile_read():
    """Per kernel class: launches, summed CUDA-event ms, algorithmic flops, bytes."""
    arr = (KernelStat * len(KCLASSES))()
    _check(load().rw_profile_read(arr, len(KCLASSES)))
    return {name: {"launches": s.launches, "ms": s.ms, "flops": s.flops, "bytes": s.bytes}
            for name, s in zip(KCLASSES, arr)}


def default_opts(**kw):
    o = Opts()
    _check(load().rw_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _nodes_desc(nodes):
    """rw_nodes from a dict of six equal-length arrays (numpy or CUDA tensors);
    returns the descriptor and the arrays it points into (kept alive)."""
    keep = []
    ptrs = []
    n = None
    for key in ("x", "y", "nx", "ny", "w", "kappa"):
        a = nodes[key]
        if not hasattr(a, "data_ptr"):
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        keep.append(a)
        ptrs.append(_ptr(a))
        m = a.numel() if hasattr(a, "numel") else a.size
        if n is not None and m != n:
            raise ValueError("node arrays must have equal lengths")
        n = m
    return NodesDesc(int(n), *ptrs), keep


class Wall:
    """Reference wall: nodes, HBS forward representation and HBS inverse."""

    def __init__(self, kind, n_panels=0, params=(), opts=None, stream=None, _handle=None, exterior=False):
        """Wall on a built-in curve; exterior=True: the exterior problem
        (rw_hbs_build_exterior: the fluid outside the curve, combined field)."""
        if _handle is not None:
            self.h = _handle
            self.n_panels = self.stats()["n_points"] // 16
            return
        L = load()
        d = WallDesc()
        d.curve_kind = {"star": CURVE_STAR, "channel": CURVE_CHANNEL}.get(kind, kind)
        d.n_panels = int(n_panels)
        for i, v in enumerate(params):
            d.params[i] = float(v)
        o = opts if opts is not None else default_opts()
        h = ctypes.c_void_p()
        build = L.rw_hbs_build_exterior if exterior else L.rw_hbs_build
        _check(build(ctypes.byref(d), ctypes.byref(o), _stream(stream), ctypes.byref(h)))
        self.h = h
        self.n_panels = int(n_panels)

    @classmethod
    def from_nodes(cls, nodes, opts=None, stream=None):
        """Wall from explicit nodes: dict x, y, nx, ny, w, kappa (16 per panel,
        panel order, counter-clockwise)."""
        desc, keep = _nodes_desc(nodes)
        o = opts if opts is not None else default_opts()
        h = ctypes.c_void_p()
        _check(load().rw_hbs_build_nodes(ctypes.byref(desc), ctypes.byref(o), _stream(stream), ctypes.byref(h)))
        del keep
        return cls(None, _handle=h)

    @classmethod
    def load(cls, path, stream=None):
        """Restore a wall written by save()."""
        h = ctypes.c_void_p()
        _check(load().rw_hbs_load(os.fsencode(path), _stream(stream), ctypes.byref(h)))
        return cls(None, _handle=h)

    def save(self, path):
        _check(load().rw_hbs_save(self.h, os.fsencode(path)))

    def stats(self):
        s = HbsStats()
        _check(load().rw_hbs_stats_get(self.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in HbsStats._fields_}

    def nodes(self, stream=None):
        n = self.stats()["n_points"]
        out = np.empty((6, n))
        _check(load().rw_hbs_nodes(self.h, _ptr(out, True), _stream(stream)))
        return dict(zip(("x", "y", "nx", "ny", "w", "kappa"), out))

    def apply_inverse(self, b, x, nrhs=1, stream=None):
        _check(load().rw_hbs_apply_inverse(self.h, nrhs, _ptr(b), _ptr(x, True), _stream(stream)))
        return x

    def apply_inverse_noalloc(self, b, x, nrhs=1, stream=None):
        """x = A_oo^{-1} b with no device allocation (device buffers only)."""
        _check(load().rw_hbs_apply_inverse_noalloc(self.h, nrhs, _ptr(b), _ptr(x, True), _stream(stream)))
        return x

    def apply_forward(self, x, y, nrhs=1, stream=None):
        _check(load().rw_hbs_apply_forward(self.h, nrhs, _ptr(x), _ptr(y, True), _stream(stream)))
        return y

    def refine(self, panels, levels, stream=None, added=None):
        """Refinement of the cut panels; added = the sub-panels' nodes (dict as
        for from_nodes, window order) instead of evaluating the wall's curve."""
        return Refinement(self, panels, levels, stream, added)

    def add_holes(self, holes, stream=None):
        """Factor the wall with holes added (App. B): holes is a list of dicts
        with cx, cy, R and optionally a, k (shape r = R (1 + a cos(k t))) and
        P (panels, default 10).  Returns a Refinement handle."""
        return Refinement(self, None, None, stream, holes=holes)

    def close(self):
        if getattr(self, "h", None):
            load().rw_hbs_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Refinement:
    """Algorithm 1 pre-computation for one modification of a Wall: a local
    refinement (cut panels split into sub-panels, Sec. 3.1) or, through
    Wall.add_holes, holes added inside the wall (App. B).  Both give the same
    handle: solve (MODE_DIRECT, MODE_DIRECT_REFINED, MODE_DIRECT_IR,
    MODE_DIRECT_IR_DF, MODE_GMRES_FP32, MODE_GMRES_BF16, MODE_GMRES_MIXED),
    apply_refined,
    stokeslet_data, pressure, nodes, Batch."""

    def __init__(self, wall, panels, levels, stream=None, added=None, holes=None):
        L = load()
        h = ctypes.c_void_p()
        if holes is not None:
            arr = (HoleDesc * len(holes))(*[HoleDesc(float(d["cx"]), float(d["cy"]), float(d["R"]),
                                                       float(d.get("a", 0.0)), int(d.get("k", 1)),
                                                       int(d.get("P", 10))) for d in holes])
            _check(L.rw_holes_factor(wall.h, len(holes), arr, _stream(stream), ctypes.byref(h)))
            self.h = h
            self.wall = wall
            return
        p = (ctypes.c_int * len(panels))(*[int(v) for v in panels])
        lv = (ctypes.c_int * len(levels))(*[int(v) for v in levels])
        if added is None:
            _check(L.rw_refine_factor(wall.h, len(panels), p, lv, _stream(stream), ctypes.byref(h)))
        else:
            desc, keep = _nodes_desc(added)
            _check(L.rw_refine_factor_nodes(wall.h, len(panels), p, lv, ctypes.byref(desc), _stream(stream),
                                            ctypes.byref(h)))
            del keep
        self.h = h
        self.wall = wall  # the wall must outlive the refinement

    def stats(self):
        s = RefStats()
        _check(load().rw_ref_stats_get(self.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in RefStats._fields_}

    def nodes(self, stream=None):
        n = self.stats()["n_n"]
        out = np.empty((6, n))
        _check(load().rw_ref_nodes(self.h, _ptr(out, True), _stream(stream)))
        return dict(zip(("x", "y", "nx", "ny", "w", "kappa"), out))

    def apply_refined(self, tau, y, nrhs=1, stream=None):
        """y = A_nn tau with the exact refined operator."""
        _check(load().rw_apply_refined(self.h, nrhs, _ptr(tau), _ptr(y, True), _stream(stream)))
        return y

    def stokeslet_data(self, src, f, g, nrhs=1, stream=None):
        """g = boundary data from point forces: src (n_src, 2), f (nrhs, n_src, 2)."""
        n_src = src.shape[0] if hasattr(src, "shape") else len(src) // 2
        _check(load().rw_stokeslet_data(self.h, n_src, _ptr(src), nrhs, _ptr(f), _ptr(g, True), _stream(stream)))
        return g

    def pressure(self, tau, targets, p, nrhs=1, stream=None):
        """p = pressure of the velocity represented by tau (the double layer;
        for holes also their single layer) at targets (nt, 2); p: (nrhs, nt)."""
        nt = targets.shape[0] if hasattr(targets, "shape") else len(targets) // 2
        _check(load().rw_pressure(self.h, nrhs, _ptr(tau), nt, _ptr(targets), _ptr(p, True), _stream(stream)))
        return p

    def solve(self, g, tau, nrhs=1, targets=None, u=None, mode=MODE_DIRECT, stream=None):
        info = Info()
        nt = 0 if targets is None else (targets.shape[0] if hasattr(targets, "shape") else len(targets) // 2)
        _check(load().rw_solve(self.h, nrhs, _ptr(g), _ptr(tau, True), nt, _ptr(targets), _ptr(u, True),
                               mode, _stream(stream), ctypes.byref(info)))
        return {"iters": info.iters, "rel_residual": info.rel_residual, "k_woodbury": info.k_woodbury,
                "cond_w": info.cond_w}

    def close(self):
        if getattr(self, "h", None):
            load().rw_ref_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def refined_points(n_panels, levels):
    """N_n for a refinement of a wall with n_panels panels."""
    return 16 * (n_panels - len(levels)) + sum(16 << int(L) for L in levels)


class Server:
    """Continuous-batching server over resident walls (C ABI rw_server_*)."""

    def __init__(self, n_workers=4, max_device_bytes=64 << 30, cache_bytes=0):
        h = ctypes.c_void_p()
        _check(load().rw_server_create(int(n_workers), int(max_device_bytes), ctypes.byref(h)))
        self.h = h
        self._keep = {}
        if cache_bytes:
            self.set_cache(cache_bytes)

    def set_cache(self, max_bytes):
        """Keep refinement factors for reuse by later requests (0 disables)."""
        _check(load().rw_server_set_cache(self.h, int(max_bytes)))

    def stats(self):
        h, m, b = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().rw_server_stats(self.h, ctypes.byref(h), ctypes.byref(m), ctypes.byref(b)))
        return {"hits": h.value, "misses": m.value, "cache_bytes": b.value}

    def submit(self, wall, panels, levels, src, f, nrhs=1, targets=None, mode=MODE_DIRECT):
        """Queue one request; returns (ticket, tau, u) with tau, u filled on completion.
        src: (n_src, 2); f: (nrhs, n_src, 2) host arrays."""
        src = np.ascontiguousarray(src, dtype=np.float64)
        f = np.ascontiguousarray(f, dtype=np.float64)
        nn = refined_points(wall.n_panels, levels)
        tau = np.empty((nrhs, 2 * nn))
        nt = 0 if targets is None else len(targets)
        tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.float64)
        u = np.empty((nrhs, 2 * nt)) if nt else None
        p = (ctypes.c_int * len(panels))(*[int(v) for v in panels])
        lv = (ctypes.c_int * len(levels))(*[int(v) for v in levels])
        q = Request(wall.h, len(panels), p, lv, int(nrhs), src.shape[0], src.ctypes.data, f.ctypes.data, nt,
                    tg.ctypes.data if nt else None, tau.ctypes.data, u.ctypes.data if nt else None, int(mode))
        t = ctypes.c_longlong()
        _check(load().rw_server_submit(self.h, ctypes.byref(q), ctypes.byref(t)))
        self._keep[t.value] = (tau, u, src, f, tg, p, lv)
        return t.value, tau, u

    def poll(self, ticket):
        st = ctypes.c_int()
        lat = ctypes.c_double(0.0)
        _check(load().rw_server_poll(self.h, ticket, ctypes.byref(st), ctypes.byref(lat)))
        return st.value, lat.value

    def wait(self, ticket):
        """Block until the request is done; returns its latency in ms."""
        lat = ctypes.c_double(0.0)
        rc = load().rw_server_wait(self.h, ticket, ctypes.byref(lat))
        self._keep.pop(ticket, None)
        _check(rc)
        return lat.value

    def close(self):
        if getattr(self, "h", None):
            load().rw_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batched single-launch solve over many refinements (C ABI rw_batch_*)."""

    def __init__(self, refs, stream=None):
        arr = (ctypes.c_void_p * len(refs))(*[r.h.value for r in refs])
        h = ctypes.c_void_p()
        _check(load().rw_batch_create(len(refs), arr, _stream(stream), ctypes.byref(h)))
        self.h = h
        self.refs = list(refs)
        off = (ctypes.c_longlong * (len(refs) + 1))()
        _check(load().rw_batch_rows(self.h, off))
        self.offsets = list(off)

    def autotune(self, nrhs=1, stream=None):
        tr = ctypes.c_int()
        ms = ctypes.c_float()
        _check(load().rw_batch_autotune(self.h, nrhs, _stream(stream), ctypes.byref(tr), ctypes.byref(ms)))
        return tr.value, ms.value

    def solve(self, g, tau, nrhs=1, use_graph=True, stream=None):
        _check(load().rw_batch_solve(self.h, nrhs, _ptr(g), _ptr(tau, True), 1 if use_graph else 0, _stream(stream)))
        return tau

    def solve_ir(self, g, tau, nrhs=1, tol=1e-10, maxit=30, stream=None):
        """Certified solve of the whole batch (rw_batch_solve_ir); returns
        {"iters", "rel_residual"}."""
        it = ctypes.c_int()
        rr = ctypes.c_double()
        _check(load().rw_batch_solve_ir(self.h, nrhs, _ptr(g), _ptr(tau, True), tol, maxit, _stream(stream),
                                        ctypes.byref(it), ctypes.byref(rr)))
        return {"iters": it.value, "rel_residual": rr.value}

    def close(self):
        if getattr(self, "h", None):
            load().rw_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

