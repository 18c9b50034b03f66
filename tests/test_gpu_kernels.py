"""GPU-vs-oracle parity of every kernel of the V cycle, called one at a time through the C ABI
(hn_band_create / hn_band_get, hn_mg_apply, hn_mg_get_inner_bands) on seeded inputs spanning
several warp-tiles and a ragged last tile (N = (2^L+1)^2 is never a multiple of the 128-node tile).

Tolerances: integer work (band layout, FP16 codes, grid transfers in FP64) is compared exactly;
floating-point products against the rounding bound of their arithmetic, 16 u sum_k |a_k x_k|
with u = 2^-53 (FP64) or 2^-24 (FP32 / FP16-band arithmetic)."""
import numpy as np
import pytest

import oracle as O
from paper_0904_4152_gb300 import inputs as I
from gpu_util import abs_spmv, coef_levels, rand_interior, require_gpu

pytestmark = pytest.mark.gpu
U64, U32 = 2.0 ** -53, 2.0 ** -24


@pytest.fixture(scope="module")
def hn():
    return require_gpu()


@pytest.mark.parametrize("L,lognormal", [(2, False), (3, True), (5, False), (5, True), (8, True),
                                         (10, False)])
def test_assembly_layout_and_values(hn, L, lognormal):
    coef = I.lognormal_coef(L, 40 + L) if lognormal else None
    A = hn.hn_band_create(L, coef)
    try:
        got = hn.hn_band_get(A)
    finally:
        hn.hn_band_destroy(A)
    ref = O.assemble(L, coef)
    np.testing.assert_array_equal(got != 0.0, ref != 0.0)          # layout: exact
    np.testing.assert_allclose(got, ref, rtol=16 * U64, atol=0)    # values: Q1 closed form vs quadrature
    n = (1 << L) + 1
    N = n * n
    for k in range(9):                                               # GPU operator is exactly symmetric
        off = (k // 3 - 1) * n + (k % 3 - 1)
        i = np.arange(max(0, -off), min(N, N - off))
        nz = got[k, i] != 0
        np.testing.assert_array_equal(got[k, i][nz], got[8 - k, i + off][nz])


def _fp16_reference(l, coef_l):
    bands = O.assemble(l, coef_l)
    s, codes = O.quantize_fp16(l, bands)
    # entries whose quotient lies within a few FP64 ulps of a binary16 rounding midpoint may
    # round either way when the FP64 band differs by an ulp between the two assemblies
    vals = bands.copy()
    vals[4] = bands.sum(axis=0)               # slot 4 holds the row sums
    q = vals / s[:, None].astype(np.float64)
    near = np.zeros_like(q, dtype=bool)
    aq = np.abs(q)
    nz = aq > 0
    e = np.floor(np.log2(aq[nz]))
    quantum = np.where(e < -14, 2.0 ** -24, 2.0 ** (e - 10))
    frac = aq[nz] / quantum
    near[nz] = np.abs(frac - np.floor(frac) - 0.5) < 1e-9
    return bands, s, codes, near


@pytest.mark.parametrize("L", [4, 7])
def test_fp16_band_codes_and_scales(hn, L):
    coef = I.lognormal_coef(L, 77)
    A = hn.hn_band_create(L, coef)
    mg = hn.hn_mg_setup(A, prec=hn.HN_PREC_FP16BAND_DC)
    hn.hn_band_destroy(A)
    try:
        for l, cl in coef_levels(L, coef).items():
            codes, scales = hn.hn_mg_get_inner_bands(mg, l, hn.HN_PREC_FP16BAND_DC)
            _, s_ref, c_ref, near = _fp16_reference(l, cl)
            np.testing.assert_array_equal(scales, s_ref)
            # a row sum that is an FP64 rounding residue of 0 quantizes to +0 or -0: same value
            codes = np.where(codes == 0x8000, 0, codes)
            c_ref = np.where(c_ref == 0x8000, 0, c_ref)
            diff = codes != c_ref
            assert not np.any(diff & ~near), (l, int(np.sum(diff & ~near)))
            assert np.all(np.abs(codes.astype(np.int64) - c_ref.astype(np.int64))[diff] == 1)
    finally:
        hn.hn_mg_destroy(mg)


@pytest.mark.parametrize("L,lognormal", [(3, False), (5, True), (8, True), (9, False)])
def test_fp64_level_kernels(hn, L, lognormal):
    coef = I.lognormal_coef(L, 90 + L) if lognormal else None
    A = hn.hn_band_create(L, coef)
    mg = hn.hn_mg_setup(A)
    hn.hn_band_destroy(A)
    omega = 0.7
    try:
        for l, cl in coef_levels(L, coef).items():
            B = O.assemble(l, cl)
            x, rhs = rand_interior(l, 1), rand_interior(l, 2)
            scale = abs_spmv(l, B, x)
            y = hn.hn_mg_apply(mg, hn.HN_OP_SPMV, l, 0, x)
            assert np.all(np.abs(y - O.spmv(l, B, x)) <= 16 * U64 * scale)
            r = hn.hn_mg_apply(mg, hn.HN_OP_DEFECT, l, 0, x, rhs)
            assert np.all(np.abs(r - O.defect(l, B, rhs, x)) <= 16 * U64 * (scale + np.abs(rhs)))
            dinv = omega / B[4]
            xj = hn.hn_mg_apply(mg, hn.HN_OP_JACOBI, l, 0, x, rhs)
            tol = 16 * U64 * ((scale + np.abs(rhs)) * dinv + np.abs(x))
            assert np.all(np.abs(xj - O.jacobi(l, B, omega, rhs, x)) <= tol)
            xz = hn.hn_mg_apply(mg, hn.HN_OP_JACOBI_ZERO, l, 0, None, rhs)
            ref = O.jacobi(l, B, omega, rhs, np.zeros_like(rhs))
            assert np.all(np.abs(xz - ref) <= 8 * U64 * np.abs(ref))
            if l > 2:
                rc = hn.hn_mg_apply(mg, hn.HN_OP_RESTRICT, l, 0, rhs)
                np.testing.assert_array_equal(rc, O.restrict(l, rhs))          # same order: exact
                ec = rand_interior(l - 1, 3)
                xp = hn.hn_mg_apply(mg, hn.HN_OP_PROLONG_ADD, l, 0, ec, x)
                np.testing.assert_array_equal(xp, O.prolong_add(l, ec, x))      # exact
            else:
                xc = hn.hn_mg_apply(mg, hn.HN_OP_COARSE, l, 0, None, rhs)
                np.testing.assert_allclose(xc, O.coarse_solve(l, B, rhs), rtol=1e-13, atol=1e-15)
        # deterministic defect norm on the finest level
        x, rhs = rand_interior(L, 5), rand_interior(L, 6)
        r, nrm = hn.hn_mg_apply(mg, hn.HN_OP_DEFECT, L, 0, x, rhs, want_norm=True)
        ref = np.linalg.norm(O.defect(L, O.assemble(L, coef), rhs, x))
        assert abs(nrm - ref) <= 1e-12 * ref
    finally:
        hn.hn_mg_destroy(mg)


def _inner_reference_bands(prec, l, cl):
    B = O.assemble(l, cl)
    if prec == "fp32":
        return B.astype(np.float32)
    s, codes = O.quantize_fp16(l, B)
    return O.dequantize_fp16(s, codes)


@pytest.mark.parametrize("staged", [0, 1])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("L", [4, 8, 10])    # staged: levels 9, 10 stream their bands by bulk copies
def test_inner_level_kernels(hn, prec, L, staged):
    if staged and L < 10:
        pytest.skip("the bulk-copy kernels serve levels with at least one chunk per SM")
    coef = I.lognormal_coef(L, 55)
    p = hn.HN_PREC_FP32_DC if prec == "fp32" else hn.HN_PREC_FP16BAND_DC
    rowsum = prec == "fp16"
    A = hn.hn_band_create(L, coef)
    mg = hn.hn_mg_setup(A, prec=p)
    hn.hn_band_destroy(A)
    hn.hn_mg_set_tuning(mg, 7, 16, 2, staged)
    omega = 0.7
    try:
        for l, cl in coef_levels(L, coef).items():
            B = _inner_reference_bands(prec, l, cl)             # float32 inner bands (oracle's)
            B64 = B.astype(np.float64)
            x = rand_interior(l, 11, np.float32)
            rhs = rand_interior(l, 12, np.float32)
            x64, rhs64 = x.astype(np.float64), rhs.astype(np.float64)
            # rounding scale of one row: every term |a_k| (|x_j| + |x_i|) (row-sum form) or |a_k x_j|
            scale = abs_spmv(l, B64, x64) + (np.abs(B64).sum(axis=0) * np.abs(x64) if rowsum else 0)
            # codes on a binary16 rounding midpoint may differ by one between the two quantizations
            slack = (2.0 ** -10 * np.abs(B64).max(axis=0) * 2 * np.abs(x64).max()) if rowsum else 0.0
            y = hn.hn_mg_apply(mg, hn.HN_OP_SPMV, l, 1, x)
            ref = O.spmv_rowsum(l, B, x) if rowsum else O.spmv(l, B64, x64)
            assert np.all(np.abs(y - ref) <= 16 * U32 * scale + slack)
            r = hn.hn_mg_apply(mg, hn.HN_OP_DEFECT, l, 1, x, rhs)
            ref = O.defect_f32(l, B, rhs, x, rowsum)
            assert np.all(np.abs(r - ref) <= 16 * U32 * (scale + np.abs(rhs64)) + slack)
            xj = hn.hn_mg_apply(mg, hn.HN_OP_JACOBI, l, 1, x, rhs)
            ref = O.jacobi_f32(l, B, omega, rhs, x, rowsum)
            diag = (B64[4] - (B64.sum(axis=0) - B64[4])) if rowsum else B64[4]
            dinv = omega / np.abs(diag)
            tol = 32 * U32 * ((scale + np.abs(rhs64)) * dinv + np.abs(x64)) + 4 * slack * dinv
            assert np.all(np.abs(xj - ref) <= tol)
            xz = hn.hn_mg_apply(mg, hn.HN_OP_JACOBI_ZERO, l, 1, None, rhs)
            ref = O.jacobi_f32(l, B, omega, rhs, np.zeros_like(x), rowsum)
            assert np.all(np.abs(xz - ref) <= 8 * U32 * np.abs(ref) + 4 * slack * dinv * np.abs(rhs64))
            if l > 2:
                rc = hn.hn_mg_apply(mg, hn.HN_OP_RESTRICT, l, 1, rhs)
                ref = O.restrict(l, rhs64)
                assert np.all(np.abs(rc - ref) <= 8 * U32 * O.restrict(l, np.abs(rhs64)))
                ec = rand_interior(l - 1, 13, np.float32)
                xp = hn.hn_mg_apply(mg, hn.HN_OP_PROLONG_ADD, l, 1, ec, x)
                ref = O.prolong_add(l, ec.astype(np.float64), x64)
                assert np.all(np.abs(xp - ref) <= 4 * U32 * (np.abs(ref) + np.abs(x64)) + 4 * U32 * np.abs(ec).max())
            else:
                xc = hn.hn_mg_apply(mg, hn.HN_OP_COARSE, l, 1, None, rhs)
                ref = O.coarse_solve(l, O.assemble(l, cl), rhs64)
                assert np.all(np.abs(xc - ref) <= 2 * U32 * np.abs(ref) + 1e-12)
    finally:
        hn.hn_mg_destroy(mg)
