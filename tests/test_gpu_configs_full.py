"""Parity at the full sizes of the benchmark configurations (Sec. 6.2 multigrid solver, Sec. 6.2.1
accuracy of the mixed scheme), through the C ABI, against the oracle.

  L = 12, lognormal coefficient (sigma 1, correlation length 0.1, field seed 0), b ~ U[-1,1]
    seed 1: FP64 V cycles in lockstep with the oracle (G1; a = 16.8 M nodes has 131,072 tiles, so
    the norms are summed in groups and the levels take the bulk-sized grids), and every precision
    solved to 1e-8 and checked with the oracle's FP64 operator (G2).
  L = 10, a = 1, b ~ U[-1,1] seed 0: the FP32-inner and FP16-band-inner defect corrections and CG
    preconditioned by one FP32 cycle, run to 1e-11, against the oracle solved to 1e-13 (G3).
  The 256-problem batch (L ~ U{5..9} seed 0, lognormal fields seeds 1000 + j, right-hand sides
    seeds 2000 + j), FP32-inner defect correction: every member checked with the oracle's operator
    (G2), and a seeded sample of 16 members solved alone gives the same bits as in the batch.
"""
import numpy as np
import pytest

import oracle as O
from paper_0904_4152_gb300 import inputs as I
from gpu_util import abs_spmv, oracle_relres, require_gpu, solve

pytestmark = pytest.mark.gpu
RELRES = 1.0001e-8


@pytest.fixture(scope="module")
def hn():
    return require_gpu()


@pytest.fixture(scope="module")
def l12():
    L = 12
    coef = I.lognormal_coef(L, 0)
    b = I.rhs_uniform(L, 1)
    return L, coef, b, O.assemble(L, coef)


def test_l12_lognormal_fp64_lockstep(hn, l12):
    L, coef, b, _ = l12
    k = 3
    x, st, status = solve(hn, L, b, coef, tol=0.0, max_cycles=k)
    assert status == hn.HN_ERR_NOT_CONVERGED and st["cycles"] == k
    xr, sr = O.mg_solve(L, b, coef=coef, tol=0.0, max_cycles=k)
    assert sr["cycles"] == k
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-9
    assert abs(st["relres"] - sr["relres"]) <= 1e-6 * sr["relres"]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_l12_lognormal_every_precision_meets_the_oracle_residual(hn, l12, prec):
    L, coef, b, A = l12
    x, st, status = solve(hn, L, b, coef, prec=prec)
    assert status == hn.HN_OK
    nb = np.linalg.norm(b)
    rel = np.linalg.norm(O.defect(L, A, b, x)) / nb
    assert rel <= RELRES
    # the solver's own FP64 residual is the oracle's up to rounding: two evaluations of b - A x
    # differ by at most 16 u (|A| |x| + |b|) per entry, so their norms by at most the norm of that
    bound = 16 * 2.0 ** -53 * np.linalg.norm(abs_spmv(L, A, x) + np.abs(b)) / nb
    assert abs(st["relres"] - rel) <= bound


@pytest.fixture(scope="module")
def l10_tight():
    L = 10
    b = I.rhs_uniform(L, 0)
    xs, ss = O.mg_solve(L, b, tol=1e-13)
    assert ss["converged"]
    return L, b, xs


@pytest.mark.parametrize("prec,solver", [(1, 0), (2, 0), (1, 1)])
def test_l10_solution_matches_the_oracle_tight_solve(hn, l10_tight, prec, solver):
    L, b, xs = l10_tight
    x, st, status = solve(hn, L, b, prec=prec, solver=solver, tol=1e-11)
    assert status == hn.HN_OK
    assert oracle_relres(L, None, b, x) <= 1.0001e-11
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-9
    # at the benchmark tolerance the same solve meets G2
    x8, st8, status = solve(hn, L, b, prec=prec, solver=solver)
    assert status == hn.HN_OK and oracle_relres(L, None, b, x8) <= RELRES


def test_batch_of_256_uneven_problems(hn):
    count = 256
    levels = [int(v) for v in I.batch_levels(count, seed=0)]
    assert min(levels) >= 5 and max(levels) <= 9
    mgs, bs, coefs = [], [], []
    try:
        for j, L in enumerate(levels):
            coef, b = I.batch_problem(j, L)
            A = hn.hn_band_create(L, coef)
            try:
                mgs.append(hn.hn_mg_setup(A, prec=hn.HN_PREC_FP32_DC))
            finally:
                hn.hn_band_destroy(A)
            bs.append(b)
            coefs.append(coef)
        xs, stats, status = hn.hn_mg_solve_batch(mgs, levels, bs)
        assert status == hn.HN_OK
        for j, L in enumerate(levels):
            assert stats[j]["status"] == hn.HN_OK
            assert oracle_relres(L, coefs[j], bs[j], xs[j]) <= RELRES, j
        rng = np.random.default_rng(2024)
        for j in sorted(rng.choice(count, size=16, replace=False)):
            xa, sa, sta = hn.hn_mg_solve(mgs[j], levels[j], bs[j])
            assert sta == hn.HN_OK
            np.testing.assert_array_equal(xs[j], xa)
            assert stats[j]["cycles"] == sa["cycles"]
            assert stats[j]["outer_iters"] == sa["outer_iters"]
    finally:
        for m in mgs:
            hn.hn_mg_destroy(m)
