"""Python view of the plain FP64 CPU oracle (``hn_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this package; the product library never does.  Each function is a thin
ctypes call into the C++ oracle, which restates the mathematics of the HONEI paper's Poisson
client (Sec. 2.1 discretisation, Sec. 6.2 multigrid and mixed-precision defect correction, CG
with a multigrid preconditioner and CG as the coarse solver).

Vectors are numpy float64 arrays of length N = (2^L+1)^2, node i = iy*n + ix.  Bands are a
(9, N) float64 array, band k holding A[i, i + dy*n + dx] with (dy, dx) = (k//3 - 1, k%3 - 1).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

PREC_FP64, PREC_FP32_DC, PREC_FP16BAND_DC, PREC_FP32_ONLY = 0, 1, 2, 3
# Dirichlet sides: bits 1 bottom (y = 0), 2 right (x = 1), 4 top (y = 1), 8 left (x = 0); the
# other sides are free Neumann
ALL_DIRICHLET, DIRICHLET_LEFT_RIGHT = 15, 10


def _sides(bc):
    if not (0 < bc <= 15):
        raise ValueError("at least one Dirichlet side (bits 1, 2, 4, 8)")
    lib().or_set_dirichlet(bc)


class Stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("inner_cycles", ctypes.c_int), ("converged", ctypes.c_int),
                ("relres", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        up = ctypes.POINTER(ctypes.c_uint16)
        L.or_n.restype = ctypes.c_long
        L.or_N.restype = ctypes.c_long
        L.or_norm2.restype = ctypes.c_double
        L.or_axpy_f32.argtypes = [ctypes.c_long, ctypes.c_float, fp, fp]
        L.or_axpy_f64.argtypes = [ctypes.c_long, ctypes.c_double, dp, dp]
        L.or_dot_f32.argtypes = [ctypes.c_long, fp, fp]
        L.or_dot_f32.restype = ctypes.c_double
        L.or_dot_f64.argtypes = [ctypes.c_long, dp, dp]
        L.or_dot_f64.restype = ctypes.c_double
        L.or_norm2.argtypes = [ctypes.c_long, dp]
        L.or_fp16_rne.restype = ctypes.c_uint16
        L.or_fp16_rne.argtypes = [ctypes.c_double]
        L.or_fp16_to_float.restype = ctypes.c_float
        L.or_fp16_to_float.argtypes = [ctypes.c_uint16]
        L.or_element_stiffness.argtypes = [ctypes.c_double, dp]
        L.or_assemble.argtypes = [ctypes.c_int, dp, dp]
        L.or_coarsen_coef.argtypes = [ctypes.c_int, dp, dp]
        L.or_spmv.argtypes = [ctypes.c_int, dp, dp, dp]
        L.or_defect.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        L.or_jacobi.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp, dp]
        L.or_restrict.argtypes = [ctypes.c_int, dp, dp]
        L.or_prolong_add.argtypes = [ctypes.c_int, dp, dp]
        L.or_coarse_solve.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int]
        L.or_coarse_solve.restype = ctypes.c_int
        L.or_quantize_fp16.argtypes = [ctypes.c_int, dp, fp, up]
        L.or_spmv_rowsum.argtypes = [ctypes.c_int, fp, fp, fp]
        L.or_defect_f32.argtypes = [ctypes.c_int, fp, fp, fp, fp, ctypes.c_int]
        L.or_jacobi_f32.argtypes = [ctypes.c_int, fp, ctypes.c_float, fp, fp, fp, ctypes.c_int]
        L.or_mg_solve.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, dp, ctypes.POINTER(Stats)]
        L.or_mg_solve.restype = ctypes.c_int
        L.or_pcg_solve.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, dp, ctypes.POINTER(Stats)]
        L.or_pcg_solve.restype = ctypes.c_int
        L.or_precondition.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp]
        L.or_precondition.restype = ctypes.c_int
        L.or_load_sinsin.argtypes = [ctypes.c_int, dp]
        L.or_l2_error_sinsin.argtypes = [ctypes.c_int, dp]
        L.or_l2_error_sinsin.restype = ctypes.c_double
        L.or_load_sincos.argtypes = [ctypes.c_int, dp]
        L.or_l2_error_sincos.argtypes = [ctypes.c_int, dp]
        L.or_l2_error_sincos.restype = ctypes.c_double
        for t, ct in (("f32", ctypes.c_float), ("f64", ctypes.c_double)):
            vp = ctypes.POINTER(ct)
            getattr(L, "or_band4_spmv_" + t).argtypes = [ctypes.c_long, ctypes.POINTER(ctypes.c_longlong),
                                                        ctypes.POINTER(vp), vp, vp]
            getattr(L, "or_swe_predict_" + t).argtypes = [ctypes.c_long, ctypes.POINTER(ctypes.c_longlong),
                                                         ctypes.POINTER(vp), vp, vp, vp, vp, vp]
        L.or_set_dirichlet.argtypes = [ctypes.c_uint]
        L.or_set_dirichlet.restype = None
        _lib = L
    return _lib


def _p(a, ctype=ctypes.c_double):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def n_of(L):
    return (1 << L) + 1


def N_of(L):
    return n_of(L) ** 2


def element_stiffness(h=1.0):
    K = np.zeros(16)
    lib().or_element_stiffness(h, _p(K))
    return K.reshape(4, 4)


def assemble(L, coef=None, bc=ALL_DIRICHLET):
    """Q1 stiffness matrix of -div(a grad u) as 9 bands, Dirichlet rows/columns eliminated."""
    bands = np.zeros((9, N_of(L)))
    c = None if coef is None else _f64(coef)
    _sides(bc)
    lib().or_assemble(L, _p(c), _p(bands))
    return bands


def coarsen_coef(Lf, coef):
    nc = n_of(Lf - 1) - 1
    out = np.zeros(nc * nc)
    lib().or_coarsen_coef(Lf, _p(_f64(coef)), _p(out))
    return out


def spmv(L, bands, x):
    y = np.zeros(N_of(L))
    lib().or_spmv(L, _p(_f64(bands)), _p(_f64(x)), _p(y))
    return y


def defect(L, bands, b, x):
    r = np.zeros(N_of(L))
    lib().or_defect(L, _p(_f64(bands)), _p(_f64(b)), _p(_f64(x)), _p(r))
    return r


def norm2(v):
    v = _f64(v)
    return lib().or_norm2(v.size, _p(v))


def jacobi(L, bands, omega, b, x):
    out = np.zeros(N_of(L))
    lib().or_jacobi(L, _p(_f64(bands)), omega, _p(_f64(b)), _p(_f64(x)), _p(out))
    return out


def restrict(Lf, rf, bc=ALL_DIRICHLET):
    rc = np.zeros(N_of(Lf - 1))
    _sides(bc)
    lib().or_restrict(Lf, _p(_f64(rf)), _p(rc))
    return rc


def prolong_add(Lf, ec, xf, bc=ALL_DIRICHLET):
    out = _f64(xf).copy()
    _sides(bc)
    lib().or_prolong_add(Lf, _p(_f64(ec)), _p(out))
    return out


def coarse_solve(Lc, bands, b, bc=ALL_DIRICHLET, cg=False, steps=False):
    """Coarsest-level solve: exact (Cholesky) or unpreconditioned CG (cg=True); with steps=True
    also returns the CG steps taken."""
    x = np.zeros(N_of(Lc))
    _sides(bc)
    rc = lib().or_coarse_solve(Lc, _p(_f64(bands)), _p(_f64(b)), _p(x), 1 if cg else 0)
    if rc < 0:
        raise ValueError("coarse matrix not positive definite")
    return (x, rc) if steps else x


def fp16_rne(v):
    """IEEE binary16 round-to-nearest-even codes (uint16) of float64 values."""
    v = np.asarray(v, dtype=np.float64)
    f = lib().or_fp16_rne
    return np.array([f(float(t)) for t in v.ravel()], dtype=np.uint16).reshape(v.shape)


def quantize_fp16(L, bands):
    s = np.zeros(9, dtype=np.float32)
    codes = np.zeros((9, N_of(L)), dtype=np.uint16)
    lib().or_quantize_fp16(L, _p(_f64(bands)), _p(s, ctypes.c_float), _p(codes, ctypes.c_uint16))
    return s, codes


def dequantize_fp16(scales, codes):
    """Float32 values s_k * float(h) of quantized band arrays."""
    return codes.view(np.float16).astype(np.float32) * np.asarray(scales, dtype=np.float32)[:, None]


def spmv_rowsum(L, deq_bands, x):
    """FP16-band inner operator in row-sum form on dequantized float32 bands (float arithmetic)."""
    y = np.zeros(N_of(L), dtype=np.float32)
    b = np.ascontiguousarray(deq_bands, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    lib().or_spmv_rowsum(L, _p(b, ctypes.c_float), _p(xx, ctypes.c_float), _p(y, ctypes.c_float))
    return y


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def defect_f32(L, bands, b, x, rowsum):
    """Float-arithmetic defect b - A x of an inner operator (rowsum: FP16 row-sum form)."""
    r = np.zeros(N_of(L), dtype=np.float32)
    fp = ctypes.c_float
    lib().or_defect_f32(L, _p(_f32(bands), fp), _p(_f32(b), fp), _p(_f32(x), fp), _p(r, fp),
                        1 if rowsum else 0)
    return r


def jacobi_f32(L, bands, omega, b, x, rowsum):
    """Float-arithmetic damped Jacobi step of an inner operator."""
    out = np.zeros(N_of(L), dtype=np.float32)
    fp = ctypes.c_float
    lib().or_jacobi_f32(L, _p(_f32(bands), fp), omega, _p(_f32(b), fp), _p(_f32(x), fp),
                        _p(out, fp), 1 if rowsum else 0)
    return out


def mg_solve(L, b, coef=None, x0=None, prec=PREC_FP64, pre=2, post=2, omega=0.7, tol=1e-8,
             max_cycles=100, max_outer=50, inner_tol=1e-2, inner_max=10, coarse_L=2,
             history=False, bc=ALL_DIRICHLET, coarse_cg=False):
    """Multigrid solve; returns (x, stats dict[, relres history])."""
    _sides(bc)
    N = N_of(L)
    x = np.zeros(N) if x0 is None else _f64(x0).copy()
    c = None if coef is None else _f64(coef)
    hlen = max(max_cycles, max_outer) + 2
    hist = np.full(hlen, np.nan) if history else None
    st = Stats()
    rc = lib().or_mg_solve(L, _p(c), _p(_f64(b)), _p(x), prec, pre, post, omega, tol,
                           max_cycles, max_outer, inner_tol, inner_max, coarse_L,
                           1 if coarse_cg else 0, _p(hist), ctypes.byref(st))
    if rc < 0:
        raise ValueError("bad arguments to the oracle solve")
    stats = dict(cycles=st.cycles, outer_iters=st.outer_iters, inner_cycles=st.inner_cycles,
                 converged=bool(st.converged), relres=st.relres)
    if history:
        return x, stats, hist[~np.isnan(hist)]
    return x, stats


def pcg_solve(L, b, coef=None, x0=None, prec=PREC_FP64, pre=2, post=2, omega=0.7, tol=1e-8,
              max_iters=100, coarse_L=2, coarse_cg=False, history=False, bc=ALL_DIRICHLET):
    """Conjugate gradients preconditioned by one V cycle (prec 0: FP64 cycle; 1 / 2: FP32 /
    FP16-band cycle on the scaled residual).  Returns (x, stats dict[, recursive relres history]);
    stats: outer_iters = CG steps, cycles = preconditioner applications, relres = true residual."""
    _sides(bc)
    N = N_of(L)
    x = np.zeros(N) if x0 is None else _f64(x0).copy()
    c = None if coef is None else _f64(coef)
    hist = np.full(max_iters + 2, np.nan) if history else None
    st = Stats()
    rc = lib().or_pcg_solve(L, _p(c), _p(_f64(b)), _p(x), prec, pre, post, omega, tol, max_iters,
                            coarse_L, 1 if coarse_cg else 0, _p(hist), ctypes.byref(st))
    if rc < 0:
        raise ValueError("bad arguments to the oracle PCG solve")
    stats = dict(cycles=st.cycles, outer_iters=st.outer_iters, inner_cycles=st.inner_cycles,
                 converged=bool(st.converged), relres=st.relres)
    if history:
        return x, stats, hist[~np.isnan(hist)]
    return x, stats


def precondition(L, r, coef=None, prec=PREC_FP64, pre=2, post=2, omega=0.7, coarse_L=2,
                 coarse_cg=False, bc=ALL_DIRICHLET):
    """z = M r: one V cycle from zero on the right-hand side r (the PCG preconditioner)."""
    _sides(bc)
    z = np.zeros(N_of(L))
    c = None if coef is None else _f64(coef)
    rc = lib().or_precondition(L, _p(c), prec, pre, post, omega, coarse_L, 1 if coarse_cg else 0,
                               _p(_f64(r)), _p(z))
    if rc < 0:
        raise ValueError("bad arguments to the oracle preconditioner")
    return z


def load_sincos(L):
    """Load vector of f = 2 pi^2 sin(pi x) cos(pi y), exact solution sin(pi x) cos(pi y):
    Dirichlet on the left and right sides (DIRICHLET_LEFT_RIGHT), free Neumann on the others."""
    b = np.zeros(N_of(L))
    _sides(DIRICHLET_LEFT_RIGHT)
    lib().or_load_sincos(L, _p(b))
    return b


def l2_error_sincos(L, x):
    return lib().or_l2_error_sincos(L, _p(_f64(x)))


def load_sinsin(L):
    """Load vector of f = 2 pi^2 sin(pi x) sin(pi y), exact solution sin(pi x) sin(pi y)."""
    b = np.zeros(N_of(L))
    _sides(ALL_DIRICHLET)
    lib().or_load_sinsin(L, _p(b))
    return b


def l2_error_sinsin(L, x):
    return lib().or_l2_error_sinsin(L, _p(_f64(x)))


def axpy(alpha, x, y):
    """y + alpha*x with one rounding per element (x, y: float32 or float64 numpy arrays; new array)."""
    out = np.array(y, copy=True)
    if x.dtype == np.float32:
        xs = np.ascontiguousarray(x, dtype=np.float32)
        lib().or_axpy_f32(len(xs), float(np.float32(alpha)),
                          xs.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    else:
        xs = np.ascontiguousarray(x, dtype=np.float64)
        lib().or_axpy_f64(len(xs), float(alpha), xs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def dot(x, y):
    """x . y summed in long double (float32 or float64 arrays of one type)."""
    if x.dtype == np.float32:
        xs, ys = np.ascontiguousarray(x, np.float32), np.ascontiguousarray(y, np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        return lib().or_dot_f32(len(xs), xs.ctypes.data_as(fp), ys.ctypes.data_as(fp))
    xs, ys = np.ascontiguousarray(x, np.float64), np.ascontiguousarray(y, np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    return lib().or_dot_f64(len(xs), xs.ctypes.data_as(dp), ys.ctypes.data_as(dp))


def _band4_args(offsets, bands, dtype):
    """offsets: (M, 4) ints; bands: (M, 4, n) arrays -> ctypes arrays (keeps the buffers alive)."""
    ct = ctypes.c_float if dtype == np.float32 else ctypes.c_double
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64).reshape(-1))
    ba = np.asarray(bands)
    bs = [np.ascontiguousarray(ba[idx], dtype=dtype) for idx in np.ndindex(ba.shape[:-1])]
    arr = (ctypes.POINTER(ct) * len(bs))(*[b.ctypes.data_as(ctypes.POINTER(ct)) for b in bs])
    return offs.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), arr, (offs, bs), ct


def band4_spmv(offsets, bands, x):
    """y_i = sum_k band_k[i] x[i + offsets[k]] over existing columns (fused multiply-adds, k in
    order): a banded matrix with four bands at arbitrary positions (Sec. 2.2, Sec. 4.1)."""
    x = np.asarray(x)
    dt = np.float32 if x.dtype == np.float32 else np.float64
    po, pb, keep, ct = _band4_args(offsets, bands, dt)
    xx = np.ascontiguousarray(x, dtype=dt)
    y = np.zeros(xx.size, dtype=dt)
    f = lib().or_band4_spmv_f32 if dt == np.float32 else lib().or_band4_spmv_f64
    f(xx.size, po, pb, _p(xx, ct), _p(y, ct))
    return y


def swe_predict(offsets, bands, u, v, w, s=None):
    """u_new = u + M1 v + M2 w + M3 u + M4 u + s, offsets (4, 4), bands (4, 4, n), in the order of
    the definition (running sum from u, one fused multiply-add per existing entry, s last)."""
    u = np.asarray(u)
    dt = np.float32 if u.dtype == np.float32 else np.float64
    po, pb, keep, ct = _band4_args(offsets, bands, dt)
    uu, vv, ww = (np.ascontiguousarray(a, dtype=dt) for a in (u, v, w))
    ss = None if s is None else np.ascontiguousarray(s, dtype=dt)
    out = np.zeros(uu.size, dtype=dt)
    f = lib().or_swe_predict_f32 if dt == np.float32 else lib().or_swe_predict_f64
    f(uu.size, po, pb, _p(uu, ct), _p(vv, ct), _p(ww, ct), _p(ss, ct), _p(out, ct))
    return out

