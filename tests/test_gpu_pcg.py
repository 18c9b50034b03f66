"""Conjugate gradients preconditioned by one V cycle, and CG as the coarse solver (Sec. 4.1
solver plugging, Sec. 6.2 coarse CG), on the GPU against the oracle through the C ABI.

Gates as for the multigrid solves: FP64 PCG in lockstep with the oracle's PCG (same number of
steps, ||dx|| / ||x|| <= 1e-9); every converged result checked with the oracle's FP64 operator
(||b - A x|| / ||b|| <= 1e-8); results bit-identical across launch shapes, alone / in a batch /
in the server, and between the one-launch solve and host-issued iterations."""
import numpy as np
import pytest

import oracle as O
from paper_0904_4152_gb300 import inputs as I
from gpu_util import oracle_relres, rand_unknowns, require_gpu, solve

pytestmark = pytest.mark.gpu
RELRES = 1.0001e-8
LR = O.DIRICHLET_LEFT_RIGHT


@pytest.fixture(scope="module")
def hn():
    return require_gpu()


def _setup(hn, L, coef, bc=15, **opts):
    A = hn.hn_band_create_bc(L, coef, bc)
    try:
        return hn.hn_mg_setup(A, **opts)
    finally:
        hn.hn_band_destroy(A)


@pytest.mark.parametrize("L,lognormal,coarse_cg", [(3, False, False), (6, True, False), (9, True, False),
                                                   (7, True, True)])
def test_pcg_fp64_lockstep(hn, L, lognormal, coarse_cg):
    coef = I.lognormal_coef(L, 400 + L) if lognormal else None
    b = I.rhs_uniform(L, 401)
    k = 4
    x, st, status = solve(hn, L, b, coef, solver=hn.HN_SOLVER_PCG, tol=0.0, max_outer=k,
                          coarse_solver=hn.HN_COARSE_CG if coarse_cg else hn.HN_COARSE_EXACT)
    assert status == hn.HN_ERR_NOT_CONVERGED
    assert st["outer_iters"] == k and st["cycles"] == k
    xr, sr = O.pcg_solve(L, b, coef=coef, tol=0.0, max_iters=k, coarse_cg=coarse_cg)
    assert sr["outer_iters"] == k
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-9


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pcg_converges(hn, prec):
    L = 10
    coef = I.lognormal_coef(L, 0)
    b = I.rhs_uniform(L, 1)
    x, st, status = solve(hn, L, b, coef, solver=hn.HN_SOLVER_PCG, prec=prec)
    assert status == hn.HN_OK
    assert oracle_relres(L, coef, b, x) <= RELRES
    _, so = O.pcg_solve(L, b, coef=coef, prec=prec)
    assert abs(so["outer_iters"] - st["outer_iters"]) <= 1
    assert st["cycles"] == st["outer_iters"]
    # PCG needs fewer cycles than the plain multigrid iteration of the same precision
    _, sm, _ = solve(hn, L, b, coef, prec=prec)
    assert st["cycles"] < sm["cycles"]


@pytest.mark.parametrize("prec", [0, 1])
def test_pcg_with_free_sides(hn, prec):
    L = 8
    b = O.load_sincos(L)
    x, st, status = solve(hn, L, b, bc=LR, solver=hn.HN_SOLVER_PCG, prec=prec, tol=1e-10,
                          coarse_solver=hn.HN_COARSE_CG)
    xr, _ = O.mg_solve(L, b, bc=LR, tol=1e-10)
    assert status == hn.HN_OK
    assert abs(O.l2_error_sincos(L, x) / O.l2_error_sincos(L, xr) - 1) < 1e-5


@pytest.mark.parametrize("coarse_L,bc,prec", [(2, 15, 0), (3, 15, 0), (4, 15, 0), (3, LR, 0),
                                              (4, 1, 1), (2, 15, 1)])
def test_coarse_cg_kernel(hn, coarse_L, bc, prec):
    L = coarse_L + 2
    coef = I.lognormal_coef(L, 90 + coarse_L)
    mg = _setup(hn, L, coef, bc, prec=prec, coarse_L=coarse_L, coarse_solver=hn.HN_COARSE_CG)
    try:
        cl = coef
        for l in range(L, coarse_L, -1):
            cl = O.coarsen_coef(l, cl)
        B = O.assemble(coarse_L, cl, bc=bc)
        rhs = rand_unknowns(coarse_L, bc, 7)
        inner = 1 if prec else 0
        xc = hn.hn_mg_apply(mg, hn.HN_OP_COARSE, coarse_L, inner, None,
                            rhs.astype(np.float32) if inner else rhs)
        ref = O.coarse_solve(coarse_L, B, rhs.astype(np.float32).astype(np.float64) if inner else rhs,
                             bc=bc, cg=True)
        tol = (4 * 2.0 ** -24 if inner else 1e-11) * np.abs(ref).max()
        assert np.all(np.abs(xc - ref) <= tol)
    finally:
        hn.hn_mg_destroy(mg)


@pytest.mark.parametrize("coarse_L", [2, 3])
def test_mg_with_coarse_cg_lockstep(hn, coarse_L):
    L = 7
    coef = I.lognormal_coef(L, 27)
    b = I.rhs_uniform(L, 28)
    x, st, status = solve(hn, L, b, coef, coarse_L=coarse_L, coarse_solver=hn.HN_COARSE_CG,
                          tol=0.0, max_cycles=3)
    xr, _ = O.mg_solve(L, b, coef=coef, coarse_L=coarse_L, coarse_cg=True, tol=0.0, max_cycles=3)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-9
    x, st, status = solve(hn, L, b, coef, coarse_L=coarse_L, coarse_solver=hn.HN_COARSE_CG, prec=1)
    assert status == hn.HN_OK and oracle_relres(L, coef, b, x) <= RELRES


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pcg_launch_shapes_and_host_iterations(hn, prec):
    L = 10
    coef, b = I.batch_problem(4, L)
    mg = _setup(hn, L, coef, prec=prec, solver=hn.HN_SOLVER_PCG)
    try:
        ref, st0, _ = hn.hn_mg_solve(mg, L, b)
        for shape in [(2, 1, 0, 0, 1, 1), (5, 16, 1, 0, 0, 0), (7, 8, 2, 1, 1, 1), (6, 16, 2, 0, 1, 0),
                      (8, 16, 1, 1, 1, 1),
                      (7, 16, 2, 0, 1, 0, 0), (4, 16, 2, 0, 1, 0, 10),
                      (7, 16, 2, 0, 1, 0, 0, 1), (4, 16, 2, 0, 1, 0, 0, 1), (6, 4, 2, 0, 1, 1, 0, 2),
                      (5, 16, 2, 0, 1, 0, 0, 2)]:
            hn.hn_mg_set_tuning(mg, *shape)
            x, st, _ = hn.hn_mg_solve(mg, L, b)
            np.testing.assert_array_equal(x, ref)
            assert st["cycles"] == st0["cycles"]
        hn.hn_mg_set_profiling(mg, True)
        x, st, _ = hn.hn_mg_solve(mg, L, b)
        names = {t["name"] for t in hn.hn_mg_kernel_times(mg)}
        hn.hn_mg_set_profiling(mg, False)
        np.testing.assert_array_equal(x, ref)
        assert {"pcg_q", "pcg_x", "pcg_dot", "pcg_p", "tail"} <= names
    finally:
        hn.hn_mg_destroy(mg)


def test_pcg_batch_and_server(hn):
    levels = [5, 7, 3, 8, 6]
    masks = [15, LR, 15, 7, 1]
    mgs, bs, coefs = [], [], []
    for j, (L, bc) in enumerate(zip(levels, masks)):
        coef = I.lognormal_coef(L, 1000 + j)
        mgs.append(_setup(hn, L, coef, bc, prec=1, solver=hn.HN_SOLVER_PCG))
        bs.append(I.rhs_uniform_bc(L, 2000 + j, bc))
        coefs.append(coef)
    try:
        xs, stats, status = hn.hn_mg_solve_batch(mgs, levels, bs)
        assert status == hn.HN_OK
        for j, (L, bc) in enumerate(zip(levels, masks)):
            xa, sa, _ = hn.hn_mg_solve(mgs[j], L, bs[j])
            np.testing.assert_array_equal(xs[j], xa)
            assert stats[j]["outer_iters"] == sa["outer_iters"]
            assert oracle_relres(L, coefs[j], bs[j], xs[j], bc=bc) <= RELRES
        srv = hn.hn_server_create(1 << 30, 3)
        try:
            tickets = [hn.hn_mg_submit(srv, L, bs[j], coefs[j], prec=1, solver=hn.HN_SOLVER_PCG,
                                       dirichlet_sides=masks[j]) for j, L in enumerate(levels)]
            for j, t in enumerate(tickets):
                status, x, st = hn.hn_mg_poll(srv, t, levels[j], timeout_ns=60_000_000_000)
                assert status == hn.HN_OK
                np.testing.assert_array_equal(x, xs[j])
            with pytest.raises(hn.HnError):     # the server's options are fixed by its first submit
                hn.hn_mg_submit(srv, 5, bs[0], coefs[0], prec=1)
        finally:
            hn.hn_server_destroy(srv)
    finally:
        for m in mgs:
            hn.hn_mg_destroy(m)


def test_pcg_guess_zero_rhs_and_arguments(hn):
    L = 6
    b = I.rhs_uniform(L, 3)
    mg = _setup(hn, L, None, prec=1, solver=hn.HN_SOLVER_PCG)
    try:
        x, st, status = hn.hn_mg_solve(mg, L, b)
        assert status == hn.HN_OK
        x1, st1, status = hn.hn_mg_solve(mg, L, b, x=x.copy(), x_is_guess=True)
        assert status == hn.HN_OK and st1["cycles"] == 0
        np.testing.assert_array_equal(x1, x)
        z, stz, status = hn.hn_mg_solve(mg, L, np.zeros_like(b), x=np.ones_like(b), x_is_guess=True)
        assert status == hn.HN_OK and np.all(z == 0)
    finally:
        hn.hn_mg_destroy(mg)
    A = hn.hn_band_create(L)
    try:
        for bad in (dict(solver=2), dict(coarse_solver=3), dict(solver=1, pre=1, post=3)):
            with pytest.raises(hn.HnError) as e:
                hn.hn_mg_setup(A, **bad)
            assert e.value.status == hn.HN_ERR_ARG
    finally:
        hn.hn_band_destroy(A)
