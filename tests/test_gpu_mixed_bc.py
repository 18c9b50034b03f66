"""Mixed boundary conditions on the GPU: zero Dirichlet values on the sides of a side mask, the
natural (free Neumann) condition on the others (Sec. 6.2.2), against the oracle through the C ABI.

Kernels are compared as in the all-Dirichlet parity tests (exact for layout and FP64 transfers,
rounding bounds for products); solves by FP64 lockstep and by the oracle's FP64 residual.
Side masks: 10 = Dirichlet at x = 0 and x = 1 (the paper's mixed test), 1 = bottom only (three
free sides), 7 = all but the left side, 5 = bottom and top."""
import numpy as np
import pytest

import oracle as O
from paper_0904_4152_gb300 import inputs as I
from gpu_util import abs_spmv, coef_levels, oracle_relres, rand_unknowns, require_gpu, solve

pytestmark = pytest.mark.gpu
U64, U32 = 2.0 ** -53, 2.0 ** -24
RELRES = 1.0001e-8
LR = O.DIRICHLET_LEFT_RIGHT


@pytest.fixture(scope="module")
def hn():
    return require_gpu()


def _setup(hn, L, coef, bc, **opts):
    A = hn.hn_band_create_bc(L, coef, bc)
    try:
        return hn.hn_mg_setup(A, **opts)
    finally:
        hn.hn_band_destroy(A)


@pytest.mark.parametrize("L,bc", [(2, 1), (3, LR), (5, 7), (5, 5), (8, LR), (9, 1)])
def test_assembly_with_side_mask(hn, L, bc):
    coef = I.lognormal_coef(L, 60 + L)
    A = hn.hn_band_create_bc(L, coef, bc)
    try:
        got = hn.hn_band_get(A)
    finally:
        hn.hn_band_destroy(A)
    ref = O.assemble(L, coef, bc=bc)
    np.testing.assert_array_equal(got != 0.0, ref != 0.0)
    np.testing.assert_allclose(got, ref, rtol=16 * U64, atol=0)
    d = ~I.unknown_mask(L, bc)                                  # Dirichlet rows: identity
    assert np.all(got[4, d] == 1.0) and np.all(got[[0, 1, 2, 3, 5, 6, 7, 8]][:, d] == 0.0)


@pytest.mark.parametrize("L,bc", [(3, LR), (6, 1), (9, 7)])
def test_fp64_level_kernels_with_side_mask(hn, L, bc):
    coef = I.lognormal_coef(L, 70 + L)
    mg = _setup(hn, L, coef, bc)
    omega = 0.7
    try:
        for l, cl in coef_levels(L, coef).items():
            B = O.assemble(l, cl, bc=bc)
            x, rhs = rand_unknowns(l, bc, 1), rand_unknowns(l, bc, 2)
            scale = abs_spmv(l, B, x)
            y = hn.hn_mg_apply(mg, hn.HN_OP_SPMV, l, 0, x)
            assert np.all(np.abs(y - O.spmv(l, B, x)) <= 16 * U64 * scale)
            r = hn.hn_mg_apply(mg, hn.HN_OP_DEFECT, l, 0, x, rhs)
            assert np.all(np.abs(r - O.defect(l, B, rhs, x)) <= 16 * U64 * (scale + np.abs(rhs)))
            xj = hn.hn_mg_apply(mg, hn.HN_OP_JACOBI, l, 0, x, rhs)
            tol = 16 * U64 * ((scale + np.abs(rhs)) * (omega / B[4]) + np.abs(x))
            assert np.all(np.abs(xj - O.jacobi(l, B, omega, rhs, x)) <= tol)
            xz = hn.hn_mg_apply(mg, hn.HN_OP_JACOBI_ZERO, l, 0, None, rhs)
            ref = O.jacobi(l, B, omega, rhs, np.zeros_like(rhs))
            assert np.all(np.abs(xz - ref) <= 8 * U64 * np.abs(ref))
            if l > 2:
                rc = hn.hn_mg_apply(mg, hn.HN_OP_RESTRICT, l, 0, rhs)
                np.testing.assert_array_equal(rc, O.restrict(l, rhs, bc=bc))
                ec = rand_unknowns(l - 1, bc, 3)
                xp = hn.hn_mg_apply(mg, hn.HN_OP_PROLONG_ADD, l, 0, ec, x)
                np.testing.assert_array_equal(xp, O.prolong_add(l, ec, x, bc=bc))
            else:
                xc = hn.hn_mg_apply(mg, hn.HN_OP_COARSE, l, 0, None, rhs)
                np.testing.assert_allclose(xc, O.coarse_solve(l, B, rhs, bc=bc), rtol=1e-12, atol=1e-14)
    finally:
        hn.hn_mg_destroy(mg)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("bc", [LR, 1])
def test_inner_level_kernels_with_side_mask(hn, prec, bc):
    L = 8
    coef = I.lognormal_coef(L, 81)
    rowsum = prec == "fp16"
    mg = _setup(hn, L, coef, bc, prec=hn.HN_PREC_FP32_DC if prec == "fp32" else hn.HN_PREC_FP16BAND_DC)
    omega = 0.7
    try:
        for l, cl in coef_levels(L, coef).items():
            B64 = O.assemble(l, cl, bc=bc)
            if prec == "fp32":
                B = B64.astype(np.float32)
            else:
                B = O.dequantize_fp16(*O.quantize_fp16(l, B64))
            Bd = B.astype(np.float64)
            x = rand_unknowns(l, bc, 11, np.float32)
            rhs = rand_unknowns(l, bc, 12, np.float32)
            x64, rhs64 = x.astype(np.float64), rhs.astype(np.float64)
            scale = abs_spmv(l, Bd, x64) + (np.abs(Bd).sum(axis=0) * np.abs(x64) if rowsum else 0)
            slack = (2.0 ** -10 * np.abs(Bd).max(axis=0) * 2 * np.abs(x64).max()) if rowsum else 0.0
            y = hn.hn_mg_apply(mg, hn.HN_OP_SPMV, l, 1, x)
            ref = O.spmv_rowsum(l, B, x) if rowsum else O.spmv(l, Bd, x64)
            assert np.all(np.abs(y - ref) <= 16 * U32 * scale + slack)
            r = hn.hn_mg_apply(mg, hn.HN_OP_DEFECT, l, 1, x, rhs)
            ref = O.defect_f32(l, B, rhs, x, rowsum)
            assert np.all(np.abs(r - ref) <= 16 * U32 * (scale + np.abs(rhs64)) + slack)
            xj = hn.hn_mg_apply(mg, hn.HN_OP_JACOBI, l, 1, x, rhs)
            ref = O.jacobi_f32(l, B, omega, rhs, x, rowsum)
            diag = (Bd[4] - (Bd.sum(axis=0) - Bd[4])) if rowsum else Bd[4]
            dinv = omega / np.abs(diag)
            tol = 32 * U32 * ((scale + np.abs(rhs64)) * dinv + np.abs(x64)) + 4 * slack * dinv
            assert np.all(np.abs(xj - ref) <= tol)
            if l > 2:
                rc = hn.hn_mg_apply(mg, hn.HN_OP_RESTRICT, l, 1, rhs)
                ref = O.restrict(l, rhs64, bc=bc)
                assert np.all(np.abs(rc - ref) <= 8 * U32 * O.restrict(l, np.abs(rhs64), bc=bc))
                ec = rand_unknowns(l - 1, bc, 13, np.float32)
                xp = hn.hn_mg_apply(mg, hn.HN_OP_PROLONG_ADD, l, 1, ec, x)
                ref = O.prolong_add(l, ec.astype(np.float64), x64, bc=bc)
                assert np.all(np.abs(xp - ref) <= 4 * U32 * (np.abs(ref) + np.abs(x64)) + 4 * U32 * np.abs(ec).max())
            else:
                xc = hn.hn_mg_apply(mg, hn.HN_OP_COARSE, l, 1, None, rhs)
                ref = O.coarse_solve(l, B64, rhs64, bc=bc)
                assert np.all(np.abs(xc - ref) <= 4 * U32 * np.abs(ref).max() + 1e-12)
    finally:
        hn.hn_mg_destroy(mg)


@pytest.mark.parametrize("L,bc", [(2, LR), (3, LR), (6, 1), (9, LR), (10, 5)])
def test_fp64_lockstep_with_side_mask(hn, L, bc):
    coef = I.lognormal_coef(L, 310 + L)
    b = I.rhs_uniform_bc(L, 311, bc)
    k = 3
    x, st, status = solve(hn, L, b, coef, bc=bc, tol=0.0, max_cycles=k)
    assert st["cycles"] == k
    xr, sr = O.mg_solve(L, b, coef=coef, tol=0.0, max_cycles=k, bc=bc)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-9
    assert np.all(x[~I.unknown_mask(L, bc)] == 0.0)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("bc", [LR, 7])
def test_solves_with_side_mask(hn, prec, bc):
    L = 10
    coef = I.lognormal_coef(L, 5)
    b = I.rhs_uniform_bc(L, 6, bc)
    x, st, status = solve(hn, L, b, coef, bc=bc, prec=prec)
    assert status == hn.HN_OK
    assert oracle_relres(L, coef, b, x, bc=bc) <= RELRES


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_manufactured_solution_with_free_sides(hn, prec):
    # u = sin(pi x) cos(pi y), a = 1: zero at x = 0, 1 and zero normal derivative at y = 0, 1;
    # the GPU solution has the oracle's discretization error
    L = 8
    b = O.load_sincos(L)
    x, st, status = solve(hn, L, b, bc=LR, prec=prec, tol=1e-10)
    xr, sr = O.mg_solve(L, b, tol=1e-10, bc=LR)
    assert status == hn.HN_OK and sr["converged"]
    e_gpu, e_or = O.l2_error_sincos(L, x), O.l2_error_sincos(L, xr)
    assert abs(e_gpu / e_or - 1) < 1e-5
    if prec == 0:
        assert st["cycles"] == sr["cycles"]


@pytest.mark.parametrize("prec", [1, 2])
def test_launch_shapes_with_side_mask(hn, prec):
    L = 10
    coef = I.lognormal_coef(L, 8)
    b = I.rhs_uniform_bc(L, 9, LR)
    mg = _setup(hn, L, coef, LR, prec=prec)
    try:
        ref, st0, _ = hn.hn_mg_solve(mg, L, b)
        for shape in [(2, 1, 0, 0, 1, 1), (5, 16, 1, 0, 0, 0), (7, 8, 2, 1, 1, 1), (7, 16, 2, 0, 0, 0),
                      (6, 4, 2, 0, 1, 1), (8, 16, 1, 1, 1, 0),
                      (7, 16, 2, 0, 1, 0, 0), (4, 16, 2, 0, 1, 0, 10),
                      (7, 16, 2, 0, 1, 0, 0, 1), (4, 16, 2, 0, 1, 0, 0, 1), (6, 4, 2, 0, 1, 1, 0, 2),
                      (5, 16, 2, 0, 1, 0, 0, 2)]:
            hn.hn_mg_set_tuning(mg, *shape)
            x, st, _ = hn.hn_mg_solve(mg, L, b)
            np.testing.assert_array_equal(x, ref)
            assert st["cycles"] == st0["cycles"]
    finally:
        hn.hn_mg_destroy(mg)


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_of_mixed_side_masks(hn, prec):
    levels = [5, 7, 3, 8, 6, 2]
    masks = [LR, 15, 1, 7, LR, 5]
    mgs, bs, coefs = [], [], []
    for j, (L, bc) in enumerate(zip(levels, masks)):
        coef = I.lognormal_coef(L, 1000 + j)
        mgs.append(_setup(hn, L, coef, bc, prec=prec))
        bs.append(I.rhs_uniform_bc(L, 2000 + j, bc))
        coefs.append(coef)
    try:
        xs, stats, status = hn.hn_mg_solve_batch(mgs, levels, bs)
        assert status == hn.HN_OK
        for j, (L, bc) in enumerate(zip(levels, masks)):
            xa, sa, _ = hn.hn_mg_solve(mgs[j], L, bs[j])
            np.testing.assert_array_equal(xs[j], xa)
            assert stats[j]["cycles"] == sa["cycles"]
            assert oracle_relres(L, coefs[j], bs[j], xs[j], bc=bc) <= RELRES
    finally:
        for m in mgs:
            hn.hn_mg_destroy(m)


def test_server_assembles_with_side_mask(hn):
    srv = hn.hn_server_create(1 << 30, 3)
    try:
        reqs = []
        for j, (L, bc) in enumerate([(6, LR), (8, 1), (5, 15), (7, 7)]):
            coef = I.lognormal_coef(L, 500 + j)
            b = I.rhs_uniform_bc(L, 600 + j, bc)
            reqs.append((hn.hn_mg_submit(srv, L, b, coef, prec=1, dirichlet_sides=bc), L, bc, coef, b))
        for t, L, bc, coef, b in reqs:
            status, x, st = hn.hn_mg_poll(srv, t, L, timeout_ns=60_000_000_000)
            assert status == hn.HN_OK
            xa, sa, _ = solve(hn, L, b, coef, bc=bc, prec=1)
            np.testing.assert_array_equal(x, xa)
            assert oracle_relres(L, coef, b, x, bc=bc) <= RELRES
    finally:
        hn.hn_server_destroy(srv)


def test_side_mask_arguments_checked(hn):
    L = 5
    for bad in (0, 16, 255):
        with pytest.raises(hn.HnError) as e:
            hn.hn_band_create_bc(L, None, bad)
        assert e.value.status == hn.HN_ERR_ARG
    # a right-hand side that is nonzero on a free side is valid; on a Dirichlet side it is not
    mg = _setup(hn, L, None, LR)
    try:
        b = I.rhs_uniform_bc(L, 1, LR)
        assert np.any(b[~I.interior_mask(L)] != 0.0)
        _, _, status = hn.hn_mg_solve(mg, L, b)
        assert status == hn.HN_OK
        n = (1 << L) + 1
        b[3 * n] = 1.0                                       # left side, x = 0
        with pytest.raises(hn.HnError) as e:
            hn.hn_mg_solve(mg, L, b)
        assert e.value.status == hn.HN_ERR_ARG
    finally:
        hn.hn_mg_destroy(mg)
    srv = hn.hn_server_create(1 << 28, 1)
    try:
        with pytest.raises(hn.HnError) as e:
            hn.hn_mg_submit(srv, L, I.rhs_uniform(L, 1), None, dirichlet_sides=0)
        assert e.value.status == hn.HN_ERR_ARG
    finally:
        hn.hn_server_destroy(srv)
