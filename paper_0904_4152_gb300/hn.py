"""Thin Python binding of the hn C ABI (include/hn.h, include/hn_profile.h).

Every function has the name of the C entry point it wraps and only marshals arguments: numpy
arrays become host pointers, CUDA torch tensors become device pointers, handles are opaque ctypes
pointers, and a non-OK status raises :class:`HnError` carrying the status and the library's message.
All computation happens in the CUDA library ``libhn.so``; if it is missing, loading fails.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# HN_DEBUG_CHECKS=1 in the environment loads the checked build (include/hn_debug.h)
LIB_PATH = os.path.join(HERE, "libhn_debug.so" if os.environ.get("HN_DEBUG_CHECKS") == "1" else "libhn.so")

HN_OK, HN_ERR_ARG, HN_ERR_OOM, HN_ERR_BUDGET, HN_ERR_CUDA = 0, 1, 2, 3, 4
HN_ERR_NOT_CONVERGED, HN_ERR_NONFINITE, HN_PENDING, HN_ERR_TIMEOUT, HN_ERR_STATE = 5, 6, 7, 8, 9
HN_PREC_FP64, HN_PREC_FP32_DC, HN_PREC_FP16BAND_DC = 0, 1, 2
HN_OP_SPMV, HN_OP_DEFECT, HN_OP_JACOBI, HN_OP_JACOBI_ZERO = 0, 1, 2, 3
HN_OP_RESTRICT, HN_OP_PROLONG_ADD, HN_OP_COARSE, HN_OP_PROLONG_JACOBI = 4, 5, 6, 7
HN_MIN_LEVEL, HN_MAX_LEVEL = 2, 14
# Dirichlet sides (the others are free Neumann): bottom y = 0, right x = 1, top y = 1, left x = 0
HN_DIRICHLET_BOTTOM, HN_DIRICHLET_RIGHT, HN_DIRICHLET_TOP, HN_DIRICHLET_LEFT = 1, 2, 4, 8
HN_DIRICHLET_ALL = 15
HN_SOLVER_MG, HN_SOLVER_PCG = 0, 1
HN_COARSE_EXACT, HN_COARSE_CG = 0, 1

STATUS_NAMES = {0: "HN_OK", 1: "HN_ERR_ARG", 2: "HN_ERR_OOM", 3: "HN_ERR_BUDGET", 4: "HN_ERR_CUDA",
                5: "HN_ERR_NOT_CONVERGED", 6: "HN_ERR_NONFINITE", 7: "HN_PENDING",
                8: "HN_ERR_TIMEOUT", 9: "HN_ERR_STATE"}

# symbols declared in include/*.h (checked by the tests against the shared library)
EXPORTS = [
    "hn_band_create", "hn_band_create_bc", "hn_band_get", "hn_band_level", "hn_band_nodes", "hn_band_destroy",
    "hn_mg_opts_default", "hn_mg_setup", "hn_mg_solve", "hn_mg_solve_batch", "hn_mg_device_bytes",
    "hn_mg_destroy", "hn_mg_apply", "hn_mg_get_inner_bands", "hn_server_create", "hn_mg_submit",
    "hn_mg_poll", "hn_server_query", "hn_server_destroy", "hn_last_error", "hn_version",
    "hn_mg_set_profiling", "hn_mg_kernel_times", "hn_mg_last_launches",
    "hn_band_defect_norm_static", "hn_mg_set_tuning", "hn_mg_get_tuning", "hn_mg_autotune",
    "hn_mg_autotune_batch", "hn_mg_time_kernel", "hn_axpy", "hn_dot", "hn_nrm2",
    "hn_band4_spmv", "hn_swe_predict", "hn_measure_fp_rates", "hn_tune_cache_lookup",
    "hn_tune_cache_store", "hn_debug_build", "hn_debug_check_mg", "hn_debug_check_band",
    "hn_debug_overwrite_guard",
]


class HnError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("coarse_L", ctypes.c_int), ("pre", ctypes.c_int), ("post", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("inner_max", ctypes.c_int), ("omega", ctypes.c_double), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("prec", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("dirichlet_sides", ctypes.c_uint), ("solver", ctypes.c_int),
                ("coarse_solver", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("inner_cycles", ctypes.c_int), ("status", ctypes.c_int),
                ("relres", ctypes.c_double), ("setup_ns", ctypes.c_longlong),
                ("solve_ns", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerInfo(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("active", ctypes.c_longlong), ("queued", ctypes.c_longlong),
                ("iterations", ctypes.c_longlong), ("bytes_in_use", ctypes.c_size_t),
                ("budget", ctypes.c_size_t), ("admit_ns", ctypes.c_longlong),
                ("schedule_ns", ctypes.c_longlong), ("iterate_ns", ctypes.c_longlong),
                ("retire_ns", ctypes.c_longlong)]


class Tuning(ctypes.Structure):
    _fields_ = [("tail_level", ctypes.c_int), ("cluster", ctypes.c_int), ("pdl", ctypes.c_int),
                ("staged", ctypes.c_int), ("dsm", ctypes.c_int), ("fuse_up", ctypes.c_int),
                ("mid", ctypes.c_int), ("sweep", ctypes.c_int)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("level", ctypes.c_int),
                ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double),
                ("bytes_per_launch", ctypes.c_double)]


_lib = None


def lib():
    """Load libhn.so (build it first with paper_0904_4152_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libhn.so not built: run `python -c \"import __graft_entry__ as g; "
                              "g.build()\"` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        L.hn_band_create.argtypes = [ip, vp, ctypes.POINTER(vp)]
        L.hn_band_create_bc.argtypes = [ip, vp, ctypes.c_uint, ctypes.POINTER(vp)]
        L.hn_band_get.argtypes = [vp, vp]
        L.hn_band_level.argtypes = [vp]
        L.hn_band_nodes.argtypes = [vp]
        L.hn_band_nodes.restype = ctypes.c_longlong
        L.hn_band_destroy.argtypes = [vp]
        L.hn_band_destroy.restype = None
        L.hn_mg_opts_default.argtypes = [ctypes.POINTER(Opts)]
        L.hn_mg_opts_default.restype = None
        L.hn_mg_setup.argtypes = [vp, ctypes.POINTER(Opts), ctypes.POINTER(vp)]
        L.hn_mg_solve.argtypes = [vp, vp, vp, ip, ip, ctypes.POINTER(Stats)]
        L.hn_mg_solve_batch.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp),
                                        ctypes.POINTER(vp), ip, ctypes.POINTER(Stats)]
        L.hn_mg_device_bytes.argtypes = [vp]
        L.hn_mg_device_bytes.restype = ctypes.c_size_t
        L.hn_mg_destroy.argtypes = [vp]
        L.hn_debug_check_mg.argtypes = [vp]
        L.hn_debug_check_band.argtypes = [vp]
        L.hn_debug_overwrite_guard.argtypes = [vp]
        L.hn_mg_destroy.restype = None
        L.hn_mg_apply.argtypes = [vp, ip, ip, ip, vp, vp, vp, dp]
        L.hn_mg_get_inner_bands.argtypes = [vp, ip, vp, ctypes.POINTER(ctypes.c_float)]
        L.hn_server_create.argtypes = [ctypes.c_size_t, ip, ctypes.POINTER(vp)]
        L.hn_mg_submit.argtypes = [vp, ip, vp, vp, ctypes.POINTER(Opts),
                                   ctypes.POINTER(ctypes.c_ulonglong)]
        L.hn_mg_poll.argtypes = [vp, ctypes.c_ulonglong, ctypes.c_longlong, vp,
                                 ctypes.POINTER(Stats)]
        L.hn_server_query.argtypes = [vp, ctypes.POINTER(ServerInfo)]
        L.hn_server_destroy.argtypes = [vp]
        L.hn_server_destroy.restype = None
        L.hn_last_error.restype = ctypes.c_char_p
        L.hn_version.restype = ctypes.c_char_p
        L.hn_mg_set_profiling.argtypes = [vp, ip]
        L.hn_mg_kernel_times.argtypes = [vp, ctypes.POINTER(KernelTime), ip]
        L.hn_band_defect_norm_static.argtypes = [vp, vp, vp, vp, vp, vp]
        L.hn_mg_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
        L.hn_mg_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
        L.hn_mg_autotune.argtypes = [vp, vp, ip, ctypes.POINTER(Tuning), dp, ip]
        L.hn_mg_autotune_batch.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp), ip,
                                           ctypes.POINTER(Tuning)]
        L.hn_mg_time_kernel.argtypes = [vp, ip, ip, ip, dp, dp]
        L.hn_mg_last_launches.argtypes = [vp]
        L.hn_mg_last_launches.restype = ctypes.c_longlong
        L.hn_axpy.argtypes = [ip, ctypes.c_longlong, ctypes.c_double, vp, vp, vp]
        L.hn_dot.argtypes = [ip, ctypes.c_longlong, vp, vp, vp, vp]
        L.hn_nrm2.argtypes = [ip, ctypes.c_longlong, vp, vp, vp]
        L.hn_band4_spmv.argtypes = [ip, ctypes.c_longlong, vp, vp, vp, vp]
        L.hn_swe_predict.argtypes = [ip, ctypes.c_longlong, vp, vp, vp, vp, vp, vp, vp]
        _lib = L
    return _lib


def _check(status):
    if status != HN_OK:
        raise HnError(status, hn_last_error())
    return status


def _host_ptr(a, dtype):
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous %s array" % np.dtype(dtype).name)
    return ctypes.c_void_p(a.ctypes.data)


def _vec_ptr(v, N):
    """(pointer, device flag) of a length-N float64 vector: numpy (host) or CUDA torch tensor."""
    if isinstance(v, np.ndarray):
        if v.size != N:
            raise ValueError("vector has %d entries, expected %d" % (v.size, N))
        return _host_ptr(v, np.float64), 0
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(v, torch.Tensor):
        if v.dtype != torch.float64 or not v.is_contiguous() or v.numel() != N:
            raise TypeError("expected a contiguous float64 tensor of %d entries" % N)
        return ctypes.c_void_p(v.data_ptr()), 1 if v.is_cuda else 0
    raise TypeError("vectors are numpy arrays or torch tensors")


def hn_last_error():
    return lib().hn_last_error().decode()


def hn_version():
    return lib().hn_version().decode()


def hn_band_create(L, cell_coef=None):
    h = ctypes.c_void_p()
    c = None
    if cell_coef is not None:
        cell_coef = np.ascontiguousarray(cell_coef, dtype=np.float64)
        if cell_coef.size != (1 << L) ** 2:
            raise ValueError("cell_coef needs (2^L)^2 entries")
        c = _host_ptr(cell_coef, np.float64)
    _check(lib().hn_band_create(L, c, ctypes.byref(h)))
    return h


def hn_band_create_bc(L, cell_coef=None, dirichlet_sides=HN_DIRICHLET_ALL):
    h = ctypes.c_void_p()
    c = None
    if cell_coef is not None:
        cell_coef = np.ascontiguousarray(cell_coef, dtype=np.float64)
        if cell_coef.size != (1 << L) ** 2:
            raise ValueError("cell_coef needs (2^L)^2 entries")
        c = _host_ptr(cell_coef, np.float64)
    _check(lib().hn_band_create_bc(L, c, dirichlet_sides, ctypes.byref(h)))
    return h


def hn_band_get(A):
    N = lib().hn_band_nodes(A)
    out = np.empty((9, N), dtype=np.float64)
    _check(lib().hn_band_get(A, _host_ptr(out, np.float64)))
    return out


def hn_band_level(A):
    return lib().hn_band_level(A)


def hn_band_nodes(A):
    return lib().hn_band_nodes(A)


def hn_band_destroy(A):
    """Free the operator; the checked build first verifies the guards around its device block and
    raises HnError if they were overwritten."""
    st = lib().hn_debug_check_band(A) if A and lib().hn_debug_build() else HN_OK
    msg = hn_last_error()
    lib().hn_band_destroy(A)
    if st != HN_OK:
        raise HnError(st, msg)


def hn_mg_opts_default(**overrides):
    o = Opts()
    lib().hn_mg_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream          # torch.cuda.Stream
        setattr(o, k, v)
    return o


def hn_mg_setup(A, opts=None, **overrides):
    if opts is None:
        opts = hn_mg_opts_default(**overrides)
    h = ctypes.c_void_p()
    _check(lib().hn_mg_setup(A, ctypes.byref(opts), ctypes.byref(h)))
    return h


def hn_mg_solve(mg, L, b, x=None, x_is_guess=False):
    """Solve A x = b.  b, x: numpy float64 (host) or CUDA torch float64 tensors of N entries.
    Returns (x, stats dict, status); status is HN_OK or HN_ERR_NOT_CONVERGED (other errors raise)."""
    N = ((1 << L) + 1) ** 2
    if x is None:
        x = np.zeros(N) if isinstance(b, np.ndarray) else b.new_zeros(N)
    pb, db = _vec_ptr(b, N)
    px, dx = _vec_ptr(x, N)
    if db != dx:
        raise ValueError("b and x must both be host or both be device vectors")
    st = Stats()
    status = lib().hn_mg_solve(mg, pb, px, 1 if x_is_guess else 0, db, ctypes.byref(st))
    if status not in (HN_OK, HN_ERR_NOT_CONVERGED):
        raise HnError(status, hn_last_error())
    return x, st.as_dict(), status


def hn_mg_solve_batch(mgs, levels, bs, xs=None):
    n = len(mgs)
    if xs is None:
        xs = [np.zeros(((1 << L) + 1) ** 2) if isinstance(b, np.ndarray) else b.new_zeros(b.numel())
              for L, b in zip(levels, bs)]
    pb, px, dev = [], [], set()
    for L, b, x in zip(levels, bs, xs):
        N = ((1 << L) + 1) ** 2
        p, d = _vec_ptr(b, N)
        q, e = _vec_ptr(x, N)
        pb.append(p.value)
        px.append(q.value)
        dev.update((d, e))
    if len(dev) != 1:
        raise ValueError("all vectors must be host or all device")
    arr = lambda v: (ctypes.c_void_p * n)(*v)
    stats = (Stats * n)()
    status = lib().hn_mg_solve_batch(arr([m.value for m in mgs]), n, arr(pb), arr(px),
                                     dev.pop(), stats)
    if status not in (HN_OK, HN_ERR_NOT_CONVERGED):
        raise HnError(status, hn_last_error())
    return xs, [s.as_dict() for s in stats], status


def hn_mg_device_bytes(mg):
    return lib().hn_mg_device_bytes(mg)


def hn_mg_destroy(mg):
    """Free the hierarchy; the checked build first verifies the guards around its device blocks and
    raises HnError if they were overwritten."""
    st = lib().hn_debug_check_mg(mg) if mg and lib().hn_debug_build() else HN_OK
    msg = hn_last_error()
    lib().hn_mg_destroy(mg)
    if st != HN_OK:
        raise HnError(st, msg)


def hn_debug_build():
    return bool(lib().hn_debug_build())


def hn_debug_check_mg(mg):
    _check(lib().hn_debug_check_mg(mg))


def hn_debug_overwrite_guard(mg):
    _check(lib().hn_debug_overwrite_guard(mg))


def hn_mg_apply(mg, op, level, inner, in1=None, in2=None, want_norm=False):
    """One solver kernel on one level; vectors are host arrays of the level's storage type
    (float64 for FP64 hierarchies, float32 for the inner levels of DC hierarchies)."""
    dt = np.float32 if inner else np.float64
    out_level = level - 1 if op == HN_OP_RESTRICT else level
    out = np.zeros(((1 << out_level) + 1) ** 2, dtype=dt)
    p1 = p2 = None
    keep = None
    if in1 is not None:
        a1 = np.ascontiguousarray(in1, dtype=dt)
        p1, keep = _host_ptr(a1, dt), (a1, keep)
    if in2 is not None:
        a2 = np.ascontiguousarray(in2, dtype=dt)
        p2, keep = _host_ptr(a2, dt), (a2, keep)
    nrm = ctypes.c_double(0.0)
    _check(lib().hn_mg_apply(mg, op, level, inner, p1, p2, _host_ptr(out, dt),
                             ctypes.byref(nrm) if want_norm else None))
    del keep
    return (out, nrm.value) if want_norm else out


def hn_band_defect_norm_static(A, x, b, r, norm, stream=None):
    """r = b - A x and ||r|| on caller-owned CUDA float64 tensors (norm: 1 element), with no device
    allocation inside the library; asynchronous on ``stream`` (a torch.cuda.Stream or None)."""
    N = lib().hn_band_nodes(A)
    ptrs = []
    for t, n in ((x, N), (b, N), (r, N), (norm, 1)):
        p, dev = _vec_ptr(t, n)
        if not dev:
            raise TypeError("x, b, r and norm must be CUDA tensors")
        ptrs.append(p)
    s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(lib().hn_band_defect_norm_static(A, *ptrs, s))


def hn_mg_get_inner_bands(mg, level, prec):
    N = ((1 << level) + 1) ** 2
    dt = np.float32 if prec == HN_PREC_FP32_DC else np.uint16
    out = np.zeros((9, N), dtype=dt)
    scales = (ctypes.c_float * 9)()
    _check(lib().hn_mg_get_inner_bands(mg, level, _host_ptr(out, dt), scales))
    return out, np.array(list(scales), dtype=np.float32)


def hn_mg_set_profiling(mg, enable):
    _check(lib().hn_mg_set_profiling(mg, 1 if enable else 0))


def hn_mg_kernel_times(mg, max_entries=256):
    buf = (KernelTime * max_entries)()
    n = lib().hn_mg_kernel_times(mg, buf, max_entries)
    return [dict(name=buf[i].name.decode(), level=buf[i].level, launches=buf[i].launches,
                 total_ms=buf[i].total_ms, bytes_per_launch=buf[i].bytes_per_launch)
            for i in range(n)]


def hn_mg_set_tuning(mg, tail_level, cluster, pdl=2, staged=0, dsm=1, fuse_up=0, mid=0, sweep=0):
    _check(lib().hn_mg_set_tuning(mg, ctypes.byref(Tuning(tail_level, cluster, pdl, staged, dsm, fuse_up, mid,
                                                          sweep))))


def hn_mg_get_tuning(mg):
    t = Tuning()
    _check(lib().hn_mg_get_tuning(mg, ctypes.byref(t)))
    return t.tail_level, t.cluster, t.pdl, t.staged, t.dsm, t.fuse_up, t.mid, t.sweep


def hn_mg_autotune(mg, b, reps=3, coarse_L=2):
    """Time every launch shape on this hierarchy, keep the fastest; returns (best, {shape: ms}),
    shapes as (tail_level, cluster, mid, sweep)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    cap = 3 * 5 * 16
    times = np.full(cap, np.nan)
    best = Tuning()
    _check(lib().hn_mg_autotune(mg, _host_ptr(b, np.float64), reps, ctypes.byref(best),
                                times.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cap))
    clusters = (1, 2, 4, 8, 16)
    modes = ((0, 0), (10, 0), (0, 1))                        # (mid, sweep) of the three forms
    rows = int(np.count_nonzero(~np.isnan(times))) // 15     # tail levels per form
    table = {}
    for i, v in enumerate(times):
        if not np.isnan(v):
            mi, k = divmod(i, 5 * rows)
            table[(coarse_L + k // 5, clusters[k % 5]) + modes[mi]] = float(v)
    return (best.tail_level, best.cluster, best.mid, best.sweep), table


def hn_mg_autotune_batch(mgs, bs, reps=2):
    """Time launch shapes on a batch (host right-hand sides), keep the fastest in every member."""
    n = len(mgs)
    bs = [np.ascontiguousarray(b, dtype=np.float64) for b in bs]
    arr = lambda v: (ctypes.c_void_p * n)(*v)
    best = Tuning()
    _check(lib().hn_mg_autotune_batch(arr([m.value for m in mgs]), n, arr([b.ctypes.data for b in bs]),
                                      reps, ctypes.byref(best)))
    return best.tail_level, best.cluster, best.pdl, best.mid


def hn_mg_time_kernel(mg, op, level, reps=20):
    """(mean ms per launch, algorithmic bytes per launch) of one solver kernel on one level."""
    ms, by = ctypes.c_double(), ctypes.c_double()
    _check(lib().hn_mg_time_kernel(mg, op, level, reps, ctypes.byref(ms), ctypes.byref(by)))
    return ms.value, by.value


def hn_tune_cache_store(path, gpu, L, prec, solver, coarse_solver, coarse_L, shape):
    """Store a launch shape (as hn_mg_get_tuning returns it; a 7-tuple has sweep 0) in the cache
    file `path`."""
    _check(lib().hn_tune_cache_store(path.encode(), gpu.encode(), L, prec, solver, coarse_solver,
                                     coarse_L, ctypes.byref(Tuning(*shape))))


def hn_tune_cache_lookup(path, gpu, L, prec, solver, coarse_solver, coarse_L):
    """The stored launch shape of the key, or None."""
    t = Tuning()
    st = lib().hn_tune_cache_lookup(path.encode(), gpu.encode(), L, prec, solver, coarse_solver,
                                    coarse_L, ctypes.byref(t))
    if st == HN_ERR_STATE:
        return None
    _check(st)
    return t.tail_level, t.cluster, t.pdl, t.staged, t.dsm, t.fuse_up, t.mid, t.sweep


class FpRates(ctypes.Structure):
    _fields_ = [("fp64_fma_per_s", ctypes.c_double), ("fp64_add_per_s", ctypes.c_double),
                ("fp64_mul_per_s", ctypes.c_double), ("fp32_fma_per_s", ctypes.c_double)]


def hn_measure_fp_rates():
    """Measured arithmetic rates of the current device (operations per second), as a dict."""
    r = FpRates()
    _check(lib().hn_measure_fp_rates(ctypes.byref(r)))
    return {k: getattr(r, k) for k, _ in FpRates._fields_}


def hn_mg_last_launches(mg):
    return lib().hn_mg_last_launches(mg)


def hn_server_create(budget_bytes, max_active):
    h = ctypes.c_void_p()
    _check(lib().hn_server_create(budget_bytes, max_active, ctypes.byref(h)))
    return h


def hn_mg_submit(srv, L, b, cell_coef=None, opts=None, **overrides):
    if opts is None:
        opts = hn_mg_opts_default(**overrides)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = None if cell_coef is None else np.ascontiguousarray(cell_coef, dtype=np.float64)
    t = ctypes.c_ulonglong()
    _check(lib().hn_mg_submit(srv, L, None if c is None else _host_ptr(c, np.float64),
                              _host_ptr(b, np.float64), ctypes.byref(opts), ctypes.byref(t)))
    return t.value


def hn_mg_poll(srv, ticket, L, timeout_ns=-1):
    """Returns (status, x or None, stats dict); HN_PENDING / HN_ERR_TIMEOUT do not raise."""
    x = np.zeros(((1 << L) + 1) ** 2)
    st = Stats()
    status = lib().hn_mg_poll(srv, ticket, timeout_ns, _host_ptr(x, np.float64), ctypes.byref(st))
    if status in (HN_PENDING, HN_ERR_TIMEOUT):
        return status, None, None
    return status, x, st.as_dict()


def hn_server_query(srv):
    info = ServerInfo()
    _check(lib().hn_server_query(srv, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def hn_server_destroy(srv):
    lib().hn_server_destroy(srv)


# ------------------------------------------------------------------ BLAS level 1 (hn_blas1.h)
HN_F32, HN_F64 = 0, 1


def _blas_vec(v):
    """(type, n, device pointer) of a contiguous CUDA float32/float64 torch tensor."""
    import torch
    if not (isinstance(v, torch.Tensor) and v.is_cuda and v.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor")
    if v.dtype == torch.float32:
        return HN_F32, v.numel(), ctypes.c_void_p(v.data_ptr())
    if v.dtype == torch.float64:
        return HN_F64, v.numel(), ctypes.c_void_p(v.data_ptr())
    raise TypeError("expected float32 or float64")


def _stream_ptr(stream):
    return ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)


def hn_axpy(alpha, x, y, stream=None):
    """y = alpha * x + y on the device (x, y: CUDA tensors of the same type and length)."""
    t, n, px = _blas_vec(x)
    t2, n2, py = _blas_vec(y)
    if (t, n) != (t2, n2):
        raise ValueError("x and y differ in type or length")
    _check(lib().hn_axpy(t, n, alpha, px, py, _stream_ptr(stream)))


def hn_dot(x, y, result, stream=None):
    """result[0] = x . y (result: a CUDA float64 tensor of at least one element)."""
    t, n, px = _blas_vec(x)
    t2, n2, py = _blas_vec(y)
    if (t, n) != (t2, n2):
        raise ValueError("x and y differ in type or length")
    _check(lib().hn_dot(t, n, px, py, ctypes.c_void_p(result.data_ptr()), _stream_ptr(stream)))


def hn_nrm2(x, result, stream=None):
    """result[0] = ||x||_2 (result: a CUDA float64 tensor of at least one element)."""
    t, n, px = _blas_vec(x)
    _check(lib().hn_nrm2(t, n, px, ctypes.c_void_p(result.data_ptr()), _stream_ptr(stream)))


# -------------------------------------- four-band matrices and the prediction step (hn_swe.h)
class Band4(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_longlong * 4), ("band", ctypes.c_void_p * 4)]


def _band4(offsets, bands, t, n):
    """An hn_band4 of 4 offsets and 4 CUDA tensors of type t and length n."""
    if len(offsets) != 4 or len(bands) != 4:
        raise ValueError("a four-band matrix needs 4 offsets and 4 bands")
    m = Band4()
    for k in range(4):
        tk, nk, pk = _blas_vec(bands[k])
        if (tk, nk) != (t, n):
            raise ValueError("band %d differs in type or length" % k)
        m.offset[k] = int(offsets[k])
        m.band[k] = pk.value
    return m


def hn_band4_spmv(offsets, bands, x, y, stream=None):
    """y = M x, M[i, i + offsets[k]] = bands[k][i] (CUDA tensors of x's type and length)."""
    t, n, px = _blas_vec(x)
    t2, n2, py = _blas_vec(y)
    if (t, n) != (t2, n2):
        raise ValueError("x and y differ in type or length")
    m = _band4(offsets, bands, t, n)
    _check(lib().hn_band4_spmv(t, n, ctypes.byref(m), px, py, _stream_ptr(stream)))


def hn_swe_predict(offsets, bands, u, v, w, s, u_new, stream=None):
    """u_new = u + M1 v + M2 w + M3 u + M4 u + s; offsets: 4 x 4 ints, bands: 4 x 4 CUDA tensors;
    s may be None."""
    t, n, pu = _blas_vec(u)
    ptrs = []
    for vec in (v, w, u_new) + (() if s is None else (s,)):
        tv, nv, pv = _blas_vec(vec)
        if (tv, nv) != (t, n):
            raise ValueError("vectors differ in type or length")
        ptrs.append(pv)
    ms = (Band4 * 4)(*[_band4(offsets[i], bands[i], t, n) for i in range(4)])
    _check(lib().hn_swe_predict(t, n, ms, pu, ptrs[0], ptrs[1], None if s is None else ptrs[3],
                                ptrs[2], _stream_ptr(stream)))

