"""Pins of the CPU oracle against what the mathematics and the paper fix (no GPU needed).

Each test checks the oracle against something other than itself: closed forms (Q1 element
matrix, eigenpairs of the constant-coefficient operator, transfer identities), an independent
dense assembly, dense LU, the O(h^2) error reduction printed in the paper's Table 1 (Sec. 6.2.1),
and numpy's IEEE float16 rounding.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_0904_4152_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------- helpers (tests)
def offsets(n):
    return [(k // 3 - 1) * n + (k % 3 - 1) for k in range(9)]


def dense_from_bands(L, bands):
    n = O.n_of(L)
    N = n * n
    A = np.zeros((N, N))
    for iy in range(n):
        for ix in range(n):
            i = iy * n + ix
            for k in range(9):
                jy, jx = iy + k // 3 - 1, ix + k % 3 - 1
                if 0 <= jx < n and 0 <= jy < n:
                    A[i, jy * n + jx] = bands[k, i]
    return A


def interior_idx(L):
    return np.flatnonzero(I.interior_mask(L))


def sin_mode(L, p, q):
    n = O.n_of(L)
    h = 1.0 / (n - 1)
    ix = np.arange(n)
    return np.outer(np.sin(q * np.pi * ix * h), np.sin(p * np.pi * ix * h)).ravel()  # [iy, ix]


def q1_eigenvalue(L, p, q):
    """Eigenvalue of the a=1 Q1 operator for sin mode (p, q): A = K1 x M1 + M1 x K1 (1D
    stiffness K1 = tridiag(-1, 2, -1)/h, mass M1 = tridiag(1, 4, 1) h/6)."""
    h = 1.0 / (O.n_of(L) - 1)
    k = lambda m: (2.0 / h) * (1.0 - math.cos(m * math.pi * h))
    mm = lambda m: (h / 3.0) * (2.0 + math.cos(m * math.pi * h))
    return k(p) * mm(q) + mm(p) * k(q)


# ------------------------------------------------------------------------ element / assembly
@pytest.mark.parametrize("h", [1.0, 1.0 / 8, 1.0 / 1024])
def test_element_stiffness_closed_form(h):
    # Q1 stiffness on a square, local nodes counter-clockwise: (1/6)[[4,-1,-2,-1], ...], no h in 2D
    ref = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    np.testing.assert_allclose(O.element_stiffness(h), ref, rtol=0, atol=4e-16)


def test_interior_stencil_closed_form():
    L = 5
    A = O.assemble(L)
    n = O.n_of(L)
    N = n * n
    for iy in range(2, n - 2):
        for ix in range(2, n - 2):
            i = iy * n + ix
            np.testing.assert_allclose(A[4, i], 8.0 / 3.0, rtol=0, atol=1e-15)
            for k in (0, 1, 2, 3, 5, 6, 7, 8):
                np.testing.assert_allclose(A[k, i], -1.0 / 3.0, rtol=0, atol=1e-15)
    # rows with no Dirichlet neighbour have row sum 0 (constants are in the kernel of -Laplace)
    inner = [iy * n + ix for iy in range(2, n - 2) for ix in range(2, n - 2)]
    assert np.max(np.abs(A[:, inner].sum(axis=0))) < 1e-14
    assert A.shape == (9, N)


def test_band_layout_exact():
    # structurally nonzero iff row and column are interior nodes (boundary rows: identity)
    for L in (2, 3, 5):
        a = I.lognormal_coef(L, 3)
        A = O.assemble(L, a)
        n = O.n_of(L)
        inner = I.interior_mask(L).reshape(n, n)
        for iy in range(n):
            for ix in range(n):
                i = iy * n + ix
                for k in range(9):
                    jy, jx = iy + k // 3 - 1, ix + k % 3 - 1
                    on = 0 <= jx < n and 0 <= jy < n
                    expect = inner[iy, ix] and on and inner[jy, jx]
                    if not inner[iy, ix]:
                        assert A[k, i] == (1.0 if k == 4 else 0.0)
                    else:
                        assert (A[k, i] != 0.0) == expect, (L, ix, iy, k)


def test_constant_coefficient_matches_kronecker_form():
    # independent dense construction: interior block = M1 (x) K1 + K1 (x) M1
    for L in (2, 3, 4):
        n = O.n_of(L)
        h = 1.0 / (n - 1)
        m = n - 2
        K1 = (2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)) / h
        M1 = (4 * np.eye(m) + np.eye(m, k=1) + np.eye(m, k=-1)) * h / 6
        ref = np.kron(M1, K1) + np.kron(K1, M1)
        idx = interior_idx(L)
        got = dense_from_bands(L, O.assemble(L))[np.ix_(idx, idx)]
        np.testing.assert_allclose(got, ref, rtol=0, atol=2e-15)


def test_variable_coefficient_matches_independent_quadrature():
    # independent assembly: hat-function gradients at 3x3 Gauss points of every cell
    L = 3
    n = O.n_of(L)
    h = 1.0 / (n - 1)
    a = I.lognormal_coef(L, 11)
    N = n * n
    ref = np.zeros((N, N))
    g = np.array([0.5 - 0.5 * math.sqrt(0.6), 0.5, 0.5 + 0.5 * math.sqrt(0.6)])
    w = np.array([5, 8, 5]) / 18.0
    for ey in range(n - 1):
        for ex in range(n - 1):
            nodes = [(ex + dx, ey + dy) for dy in (0, 1) for dx in (0, 1)]
            for qy in range(3):
                for qx in range(3):
                    x = (ex + g[qx]) * h
                    y = (ey + g[qy]) * h
                    grads = []
                    for (jx, jy) in nodes:
                        tx, ty = x - jx * h, y - jy * h
                        hx, hy = 1 - abs(tx) / h, 1 - abs(ty) / h
                        grads.append((-np.sign(tx) / h * hy, -np.sign(ty) / h * hx))
                    for p, (ix, iy) in enumerate(nodes):
                        for q, (jx, jy) in enumerate(nodes):
                            ref[iy * n + ix, jy * n + jx] += (w[qx] * w[qy] * h * h * a[ey * (n - 1) + ex]
                                                              * (grads[p][0] * grads[q][0] + grads[p][1] * grads[q][1]))
    idx = interior_idx(L)
    got = dense_from_bands(L, O.assemble(L, a))[np.ix_(idx, idx)]
    np.testing.assert_allclose(got, ref[np.ix_(idx, idx)], rtol=1e-13, atol=1e-14)


def test_coefficient_scaling():
    L = 4
    c = 3.25
    N1 = O.assemble(L)
    Nc = O.assemble(L, np.full((O.n_of(L) - 1) ** 2, c))
    idx = interior_idx(L)
    np.testing.assert_allclose(Nc[:, idx], c * N1[:, idx], rtol=1e-15, atol=0)


@pytest.mark.parametrize("L", [2, 3, 4, 5])
def test_symmetric_positive_definite(L):
    a = I.lognormal_coef(L, 5)
    A = O.assemble(L, a)
    n = O.n_of(L)
    N = n * n
    offs = offsets(n)
    for k in range(9):
        for i in range(N):
            j = i + offs[k]
            if 0 <= j < N and A[k, i] != 0.0:
                assert A[k, i] == A[8 - k, j]          # bit-exact symmetry
    D = dense_from_bands(L, A)
    np.linalg.cholesky(D)                              # raises if not SPD
    assert np.linalg.eigvalsh(D).min() > 0


def test_coarsen_coef_linear_field():
    # mean of 4 children of a linear field sampled at cell centres = value at the coarse centre
    Lf = 5
    nf = 1 << Lf
    c = (np.arange(nf) + 0.5) / nf
    X, Y = np.meshgrid(c, c)
    af = (2.0 + 0.7 * X - 0.3 * Y).ravel()
    nc = nf // 2
    cc = (np.arange(nc) + 0.5) / nc
    Xc, Yc = np.meshgrid(cc, cc)
    np.testing.assert_allclose(O.coarsen_coef(Lf, af), (2.0 + 0.7 * Xc - 0.3 * Yc).ravel(),
                               rtol=0, atol=1e-14)


# -------------------------------------------------------------- band operators (a = 1 modes)
@pytest.mark.parametrize("L,p,q", [(4, 1, 1), (4, 3, 7), (5, 2, 13), (5, 31, 1)])
def test_spmv_eigenpairs(L, p, q):
    A = O.assemble(L)
    v = sin_mode(L, p, q)
    lam = q1_eigenvalue(L, p, q)
    tol = 1e-14 * max(1.0, lam)
    np.testing.assert_allclose(O.spmv(L, A, v), lam * v, rtol=0, atol=tol)
    # defect of the exact eigen-solution vanishes; defect of 0 is b
    np.testing.assert_allclose(O.defect(L, A, lam * v, v), 0.0, atol=tol)
    np.testing.assert_array_equal(O.defect(L, A, v, np.zeros_like(v)), v)


@pytest.mark.parametrize("omega", [0.7, 0.5])
def test_jacobi_error_propagation(omega):
    # with b = 0 one damped Jacobi step multiplies mode (p,q) by 1 - omega * lambda / (8/3)
    L = 5
    A = O.assemble(L)
    for p, q in [(1, 1), (5, 9), (30, 30)]:
        v = sin_mode(L, p, q)
        x1 = O.jacobi(L, A, omega, np.zeros_like(v), v)
        fac = 1.0 - omega * q1_eigenvalue(L, p, q) * 3.0 / 8.0
        np.testing.assert_allclose(x1, fac * v, rtol=0, atol=1e-14)


def test_jacobi_fixed_point():
    L = 4
    a = I.lognormal_coef(L, 2)
    A = O.assemble(L, a)
    idx = interior_idx(L)
    D = dense_from_bands(L, A)
    b = I.rhs_uniform(L, 4)
    xs = np.zeros_like(b)
    xs[idx] = np.linalg.solve(D[np.ix_(idx, idx)], b[idx])
    np.testing.assert_allclose(O.jacobi(L, A, 0.7, b, xs), xs, rtol=0, atol=1e-13)


# ------------------------------------------------------------------------------ transfers
@pytest.mark.parametrize("Lf,p,q", [(4, 1, 1), (4, 3, 5), (6, 7, 30)])
def test_restriction_of_modes(Lf, p, q):
    # full weighting of a fine sin mode = (1+cos(p pi h))(1+cos(q pi h)) x the coarse mode
    hf = 1.0 / (O.n_of(Lf) - 1)
    fac = (1 + math.cos(p * math.pi * hf)) * (1 + math.cos(q * math.pi * hf))
    rc = O.restrict(Lf, sin_mode(Lf, p, q))
    np.testing.assert_allclose(rc, fac * sin_mode(Lf - 1, p, q), rtol=0, atol=1e-13)


def test_restriction_of_constant():
    Lf = 5
    rc = O.restrict(Lf, I.interior_mask(Lf).astype(float)).reshape(O.n_of(Lf - 1), -1)
    np.testing.assert_array_equal(rc[2:-2, 2:-2], 4.0)     # 1 + 4 * 1/2 + 4 * 1/4
    assert np.all(rc[0, :] == 0) and np.all(rc[:, -1] == 0)


def test_prolongation_reproduces_bilinear():
    Lf = 5
    nf, nc = O.n_of(Lf), O.n_of(Lf - 1)
    f = lambda x, y: 0.3 + 1.7 * x - 0.4 * y + 2.2 * x * y
    Xc, Yc = np.meshgrid(np.linspace(0, 1, nc), np.linspace(0, 1, nc))
    ec = (f(Xc, Yc) * I.interior_mask(Lf - 1).reshape(nc, nc)).ravel()
    xf = O.prolong_add(Lf, ec, np.zeros(nf * nf)).reshape(nf, nf)
    Xf, Yf = np.meshgrid(np.linspace(0, 1, nf), np.linspace(0, 1, nf))
    np.testing.assert_allclose(xf[2:-2, 2:-2], f(Xf, Yf)[2:-2, 2:-2], rtol=0, atol=1e-14)
    assert np.all(xf[0, :] == 0) and np.all(xf[:, 0] == 0)


def test_restriction_is_adjoint_of_prolongation():
    Lf = 6
    rng = np.random.default_rng(0)
    r = rng.standard_normal(O.N_of(Lf)) * I.interior_mask(Lf)
    e = rng.standard_normal(O.N_of(Lf - 1)) * I.interior_mask(Lf - 1)
    lhs = O.restrict(Lf, r) @ e
    rhs = r @ O.prolong_add(Lf, e, np.zeros(O.N_of(Lf)))
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(r).sum() + 1)


@pytest.mark.parametrize("Lf", [3, 4])
def test_galerkin_equals_rediscretisation(Lf):
    # for a = 1, P^T A_f P equals the re-assembled coarse operator
    Nc = O.N_of(Lf - 1)
    ic = interior_idx(Lf - 1)
    P = np.zeros((O.N_of(Lf), ic.size))
    for c, C in enumerate(ic):
        e = np.zeros(Nc)
        e[C] = 1.0
        P[:, c] = O.prolong_add(Lf, e, np.zeros(O.N_of(Lf)))
    Af = dense_from_bands(Lf, O.assemble(Lf))
    Ac = dense_from_bands(Lf - 1, O.assemble(Lf - 1))[np.ix_(ic, ic)]
    np.testing.assert_allclose(P.T @ Af @ P, Ac, rtol=0, atol=2e-15)


def test_coarse_solve_matches_dense():
    L = 2
    a = I.lognormal_coef(L, 9)
    A = O.assemble(L, a)
    b = I.rhs_uniform(L, 1)
    idx = interior_idx(L)
    ref = np.zeros_like(b)
    ref[idx] = np.linalg.solve(dense_from_bands(L, A)[np.ix_(idx, idx)], b[idx])
    np.testing.assert_allclose(O.coarse_solve(L, A, b), ref, rtol=1e-14, atol=1e-15)


# ------------------------------------------------------------------------------- multigrid
@pytest.mark.parametrize("L,lognormal", [(3, False), (4, False), (4, True)])
def test_mg_matches_dense_lu(L, lognormal):
    a = I.lognormal_coef(L, 21) if lognormal else None
    A = O.assemble(L, a)
    b = I.rhs_uniform(L, 22)
    idx = interior_idx(L)
    xs = np.zeros_like(b)
    xs[idx] = np.linalg.solve(dense_from_bands(L, A)[np.ix_(idx, idx)], b[idx])
    x, st = O.mg_solve(L, b, coef=a, tol=1e-13)
    assert st["converged"] and st["relres"] <= 1e-13
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-11


def bilinear_P(Lf):
    """Dense interpolation from level Lf - 1 to Lf, written from the bilinear definition: a fine
    node takes its coarse parent's value (even index), the mean of its two parents (odd index),
    per axis, the weights multiplying; rows of fine boundary nodes and columns of coarse boundary
    nodes are zero."""
    nf, nc = O.n_of(Lf), O.n_of(Lf - 1)
    P = np.zeros((nf * nf, nc * nc))

    def parents(f):
        return [(f // 2, 1.0)] if f % 2 == 0 else [((f - 1) // 2, 0.5), ((f + 1) // 2, 0.5)]

    for fy in range(1, nf - 1):
        for fx in range(1, nf - 1):
            for Cy, wy in parents(fy):
                for Cx, wx in parents(fx):
                    if 0 < Cx < nc - 1 and 0 < Cy < nc - 1:
                        P[fy * nf + fx, Cy * nc + Cx] += wx * wy
    return P


def dense_vcycle(L, Lc, coef, b, pre, post, omega):
    """One V(pre, post) cycle from zero in dense matrices: damped Jacobi pre-smoothing, the defect
    restricted by P^T, the same cycle on the coarser level (an exact solve on the unknowns of the
    coarsest), prolongation of the correction, post-smoothing."""
    cf = {L: coef}
    for l in range(L, Lc, -1):
        cf[l - 1] = None if cf[l] is None else O.coarsen_coef(l, cf[l])
    A = {l: dense_from_bands(l, O.assemble(l, cf[l])) for l in range(Lc, L + 1)}

    def cycle(l, rhs):
        if l == Lc:
            idx = interior_idx(l)
            x = np.zeros(rhs.size)
            x[idx] = np.linalg.solve(A[l][np.ix_(idx, idx)], rhs[idx])
            return x
        D = np.diag(A[l])
        x = np.zeros(rhs.size)
        for _ in range(pre):
            x = x + omega * (rhs - A[l] @ x) / D
        P = bilinear_P(l)
        x = x + P @ cycle(l - 1, P.T @ (rhs - A[l] @ x))
        for _ in range(post):
            x = x + omega * (rhs - A[l] @ x) / D
        return x

    return cycle(L, b)


@pytest.mark.parametrize("pre,post", [(1, 2), (2, 1), (0, 1), (2, 2)])
@pytest.mark.parametrize("L,lognormal", [(3, False), (4, True)])
def test_one_cycle_equals_its_dense_composition(L, lognormal, pre, post):
    # the cycle's structure, with unequal smoothing counts: a swapped pre/post count, a missing
    # restriction of the defect or a correction applied before the coarse solve all change it
    a = I.lognormal_coef(L, 31) if lognormal else None
    b = I.rhs_uniform(L, 32)
    z = O.precondition(L, b, coef=a, prec=O.PREC_FP64, pre=pre, post=post, omega=0.7, coarse_L=2)
    ref = dense_vcycle(L, 2, a, b, pre, post, 0.7)
    assert np.linalg.norm(z - ref) <= 1e-13 * np.linalg.norm(ref)


def test_mg_contraction_level_independent():
    # Sec. 6.2: two V(2,2) cycles gain (at least) one digit; the rate does not grow with L
    rates = []
    for L in (4, 6, 8):
        _, st, h = O.mg_solve(L, O.load_sinsin(L), tol=1e-12, history=True)
        r = h[2:6] / h[1:5]
        rates.append(r.max())
        assert st["converged"]
    assert max(rates) < 10 ** -0.5
    assert max(rates) / min(rates) < 1.5


def _golden(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if not l.startswith("#")]
    return {int(r[0]): float(r[2]) for r in rows}


@pytest.mark.slow
def test_l2_error_reduction_matches_table1():
    # Table 1: the L2 error falls by 4.00 (+-0.02) per level for L >= 5 in double and mixed
    # precision.  Our manufactured solution is sin(pi x) sin(pi y) (the paper's polynomial is
    # unnamed), so only the reduction factors are compared.
    gd, gm = _golden("table1_double_reduction.txt"), _golden("table1_mixed_reduction.txt")
    err64, err32 = {}, {}
    for L in range(4, 10):
        b = O.load_sinsin(L)
        x, st = O.mg_solve(L, b, tol=1e-11)
        err64[L] = O.l2_error_sinsin(L, x)
        x, st = O.mg_solve(L, b, prec=O.PREC_FP32_DC, tol=1e-11)
        assert st["converged"]
        err32[L] = O.l2_error_sinsin(L, x)
    for L in range(5, 10):
        assert abs(err64[L - 1] / err64[L] - gd[L]) < 0.05, (L, err64[L - 1] / err64[L])
        assert abs(err32[L - 1] / err32[L] - gm[L]) < 0.05
        assert abs(err32[L] / err64[L] - 1) < 0.01        # mixed = double accuracy


def test_l2_error_of_zero_and_of_interpolant():
    # ||sin(pi x) sin(pi y)||_L2 = 1/2; the nodal interpolant's error falls like h^2
    assert abs(O.l2_error_sinsin(5, np.zeros(O.N_of(5))) - 0.5) < 1e-10
    e = [O.l2_error_sinsin(L, sin_mode(L, 1, 1)) for L in (4, 5, 6)]
    assert 3.9 < e[0] / e[1] < 4.1 and 3.9 < e[1] / e[2] < 4.1


def test_load_vector_consistent_with_point_values():
    # b_i / (h^2 f(x_i)) -> 1 at interior nodes (f smooth, basis integrates to h^2)
    L = 7
    n = O.n_of(L)
    h = 1.0 / (n - 1)
    b = O.load_sinsin(L).reshape(n, n)
    f = 2 * np.pi ** 2 * sin_mode(L, 1, 1).reshape(n, n)
    ratio = b[1:-1, 1:-1] / (h * h * f[1:-1, 1:-1])
    assert np.max(np.abs(ratio - 1)) < 1e-3
    assert np.all(b[0, :] == 0) and np.all(b[:, -1] == 0)


@pytest.mark.parametrize("L", [4, 6])
def test_load_vector_matches_the_exact_integral(L):
    # f = 2 pi^2 sin(pi x) g(y) against the hat function of node (x_i, y_j) separates; per axis
    # the integral of sin (or cos) times a hat of half-width h is sin(pi x_i) * 2 (1 - cos pi h) /
    # (pi^2 h), and half of that (times cos(pi y_j)) for the half hat of a free side's node
    n = O.n_of(L)
    h = 1.0 / (n - 1)
    c = 2.0 * (1.0 - math.cos(math.pi * h)) / (math.pi ** 2 * h)
    x = np.arange(n) * h
    sx = np.sin(np.pi * x) * c
    exact = 2 * np.pi ** 2 * np.outer(sx, sx)                                  # [y, x]
    exact[0, :] = exact[-1, :] = exact[:, 0] = exact[:, -1] = 0.0
    b = O.load_sinsin(L).reshape(n, n)
    assert np.abs(b - exact).max() <= 1e-8 * np.abs(exact).max()
    cy = np.cos(np.pi * x) * c
    cy[0] *= 0.5
    cy[-1] *= 0.5
    exact = 2 * np.pi ** 2 * np.outer(cy, sx)                                  # Dirichlet x = 0, 1
    exact[:, 0] = exact[:, -1] = 0.0
    b = O.load_sincos(L).reshape(n, n)
    assert np.abs(b - exact).max() <= 1e-8 * np.abs(exact).max()


def test_fp16_decoding_matches_ieee():
    # every binary16 code decodes to the value numpy's IEEE half type gives it
    codes = np.arange(1 << 16, dtype=np.uint16)
    want = codes.view(np.float16).astype(np.float32)
    f = O.lib().or_fp16_to_float
    got = np.array([f(int(c)) for c in codes], dtype=np.float32)
    nan = np.isnan(want)
    assert (np.isnan(got) == nan).all()
    np.testing.assert_array_equal(got[~nan], want[~nan])
    assert (np.signbit(got[~nan]) == np.signbit(want[~nan])).all()


@pytest.mark.parametrize("prec", [O.PREC_FP32_DC, O.PREC_FP16BAND_DC])
def test_mixed_precision_reaches_fp64_tolerance(prec):
    L = 7
    a = I.lognormal_coef(L, 0)
    b = I.rhs_uniform(L, 1)
    x, st = O.mg_solve(L, b, coef=a, prec=prec)
    assert st["converged"] and st["relres"] <= 1e-8
    r = O.defect(L, O.assemble(L, a), b, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
    assert st["outer_iters"] >= 2 and st["inner_cycles"] >= st["outer_iters"]


@pytest.mark.parametrize("prec", [O.PREC_FP64, O.PREC_FP32_DC, O.PREC_FP16BAND_DC])
def test_stopping_rule_is_the_first_iterate_within_tolerance(prec):
    # the solve stops at the first cycle (FP64) or outer step (defect correction) whose FP64
    # relative residual is at most tol, and counts one entry per cycle / step
    L = 6
    a = I.lognormal_coef(L, 3)
    b = I.rhs_uniform(L, 4)
    for tol in (1e-3, 1e-5, 1e-7, 1e-9, 1e-11):
        x, st, hist = O.mg_solve(L, b, coef=a, prec=prec, tol=tol, history=True)
        assert st["converged"] and hist[-1] <= tol and (hist[:-1] > tol).all()
        steps = st["cycles"] if prec == O.PREC_FP64 else st["outer_iters"]
        assert hist.size == steps + 1
        r = O.defect(L, O.assemble(L, a), b, x)
        assert abs(np.linalg.norm(r) / np.linalg.norm(b) - hist[-1]) <= 1e-6 * hist[-1]


@pytest.mark.parametrize("inner_max", [1, 3])
def test_inner_cycles_per_outer_step_are_capped(inner_max):
    # with an inner tolerance no cycle meets, every outer step runs exactly inner_max cycles
    L = 5
    b = I.rhs_uniform(L, 5)
    x, st = O.mg_solve(L, b, prec=O.PREC_FP32_DC, inner_tol=1e-30, inner_max=inner_max,
                       max_outer=4, tol=1e-30)
    assert st["outer_iters"] == 4 and st["inner_cycles"] == 4 * inner_max


def test_inner_solve_stops_like_the_fp32_solve_of_the_scaled_defect():
    # from x = 0 the first outer step's inner solve is FP32 multigrid on d / ||d|| = b / ||b||
    # from zero, stopped at the first cycle whose FP32 residual is within inner_tol of that
    # right-hand side: the same count as the FP32-only solve of it to tol = inner_tol
    L = 6
    a = I.lognormal_coef(L, 7)
    b = I.rhs_uniform(L, 8)
    dhat = (b / np.linalg.norm(b)).astype(np.float32).astype(np.float64)
    counts = []
    for inner_tol in (0.3, 0.1, 3e-2, 1e-2, 1e-3):
        _, st = O.mg_solve(L, b, coef=a, prec=O.PREC_FP32_DC, inner_tol=inner_tol, inner_max=50,
                           max_outer=1, tol=1e-30)
        _, s32 = O.mg_solve(L, dhat, coef=a, prec=O.PREC_FP32_ONLY, tol=inner_tol, max_cycles=50)
        assert st["inner_cycles"] == s32["cycles"]
        counts.append(st["inner_cycles"])
    assert counts == sorted(counts) and counts[-1] > counts[0]


def test_fp32_only_loses_accuracy():
    # Table 1 single-precision column: pure FP32 multigrid stops improving; the error grows again
    # with the level and falls behind FP64 by more than an order of magnitude
    errs = {}
    for L in (7, 9):
        b = O.load_sinsin(L)
        x, _ = O.mg_solve(L, b, prec=O.PREC_FP32_ONLY, max_cycles=30)
        x64, _ = O.mg_solve(L, b)
        errs[L] = (O.l2_error_sinsin(L, x), O.l2_error_sinsin(L, x64))
    assert errs[9][0] > errs[7][0]
    assert errs[9][0] > 10 * errs[9][1]


# ------------------------------------------------------------------------- FP16 band storage
def test_fp16_rne_matches_ieee():
    rng = np.random.default_rng(1)
    vals = np.concatenate([
        rng.standard_normal(2000),
        rng.standard_normal(500) * 2.0 ** -16,                     # subnormal range
        rng.uniform(-1, 1, 500) * 60000.0,
        (1 + np.arange(0, 64) * 2.0 ** -11),                       # exact ties at 1
        -(2.0 ** -14) * (1 + np.arange(0, 64) * 2.0 ** -11),
        np.arange(0, 40) * 2.0 ** -25,                              # subnormal ties
        [0.0, -0.0, 1.0, -1.0, 65504.0, 2.0 ** -24],
    ])
    ref = vals.astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(O.fp16_rne(vals), ref)


@pytest.mark.parametrize("L", [5, 9])
def test_quantize_fp16_bands(L):
    # slot 4 holds the row sums; every array has its own max-abs scale; codes are numpy's RNE of
    # the FP64 quotient (at L = 9, 2.4 million values: a quotient rounded to FP32 first would
    # round about a hundred of them twice and differ)
    A = O.assemble(L, I.lognormal_coef(L, 3))
    s, codes = O.quantize_fp16(L, A)
    V = A.copy()
    V[4] = A.sum(axis=0)                      # row sums (numpy's pairwise order: agree to rounding)
    np.testing.assert_allclose(s, np.abs(V).max(axis=1).astype(np.float32), rtol=2 ** -23)
    ref = (V / s[:, None].astype(np.float64)).astype(np.float16).view(np.uint16)
    diff = codes != ref
    # a row sum may differ by an FP64 rounding from numpy's, moving a code by one at most
    assert diff[[0, 1, 2, 3, 5, 6, 7, 8]].sum() == 0
    assert np.all(np.abs(codes[4].astype(int) - ref[4].astype(int)) <= 1)
    dec = O.dequantize_fp16(s, codes).astype(np.float64)
    big = np.abs(V) > 2.0 ** -14 * s[:, None]
    assert np.all(np.abs(dec - V)[big] <= 2.0 ** -11 * np.abs(V)[big] * (1 + 1e-6))


def test_fp16_rowsum_operator_keeps_constants_in_the_kernel():
    # rows with no Dirichlet neighbour have row sum 0: the quantized operator maps constants to
    # exactly 0 there, and agrees with the FP64 9-band product to the FP16 quantum elsewhere
    L = 6
    A = O.assemble(L, I.lognormal_coef(L, 8))
    s, codes = O.quantize_fp16(L, A)
    D = O.dequantize_fp16(s, codes)
    n = O.n_of(L)
    ones = I.interior_mask(L).astype(np.float32)
    y = O.spmv_rowsum(L, D, ones).reshape(n, n)
    assert np.all(y[2:-2, 2:-2] == 0.0)
    x = np.random.default_rng(0).uniform(-1, 1, O.N_of(L)).astype(np.float32) * I.interior_mask(L)
    ref = O.spmv(L, A, x.astype(np.float64))
    scale = O.spmv(L, np.abs(A), np.abs(x.astype(np.float64)))
    assert np.all(np.abs(O.spmv_rowsum(L, D, x) - ref) <= 2.0 ** -10 * scale + 1e-6)


@pytest.mark.slow
def test_fp16_defect_correction_converges_at_large_level():
    # with the couplings quantized and the row sums kept, FP16-band defect correction contracts
    # at a level where per-entry quantization of all 9 bands would stall (perturbation >> lambda_min)
    L = 9
    a = I.lognormal_coef(L, 0)
    b = I.rhs_uniform(L, 1)
    x, st = O.mg_solve(L, b, coef=a, prec=O.PREC_FP16BAND_DC)
    assert st["converged"] and st["outer_iters"] <= 12


# ------------------------------------------------------------------ BLAS level 1 (Sec. 6.1)
def test_oracle_dot_closed_form_and_exact_sum():
    import math
    n = 1_000_000
    x = np.arange(n, dtype=np.float64)
    assert O.dot(x, np.ones(n)) == n * (n - 1) / 2                    # exact integer sum
    rng = np.random.default_rng(3)
    a, b = rng.uniform(-1, 1, 4099).astype(np.float32), rng.uniform(-1, 1, 4099).astype(np.float32)
    prods = a.astype(np.float64) * b.astype(np.float64)              # exact for float32 inputs
    exact = math.fsum(prods.tolist())                                # correctly rounded sum
    assert abs(O.dot(a, b) - exact) <= 2.0 ** -52 * abs(exact)


def test_oracle_axpy_single_rounding():
    rng = np.random.default_rng(4)
    x, y = rng.uniform(-1, 1, 5000).astype(np.float32), rng.uniform(-1, 1, 5000).astype(np.float32)
    a = np.float32(-0.37)
    # a*x + y exactly in extended precision, rounded once to float32
    ref = (np.longdouble(a) * x.astype(np.longdouble) + y.astype(np.longdouble)).astype(np.float32)
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip("no extended precision long double on this host")
    np.testing.assert_array_equal(O.axpy(a, x, y), ref)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    assert np.array_equal(O.axpy(2.0, np.ones(3), np.ones(3)), np.full(3, 3.0))
    assert np.all(np.abs(O.axpy(0.5, xd, yd) - (0.5 * xd + yd)) <= 2.0 ** -53 * (np.abs(0.5 * xd) + np.abs(yd)))


# ---------------------------------------- mixed free-Neumann / Dirichlet boundaries (Sec. 6.2.2)
LR = O.DIRICHLET_LEFT_RIGHT          # Dirichlet at x = 0, 1; free Neumann at y = 0, 1


def _unknown_mask(L, bc):
    n = (1 << L) + 1
    m = np.ones((n, n), dtype=bool)
    if bc & 1: m[0, :] = False
    if bc & 2: m[:, -1] = False
    if bc & 4: m[-1, :] = False
    if bc & 8: m[:, 0] = False
    return m.ravel()


@pytest.mark.parametrize("bc", [LR, 1, 7, 8])
def test_mixed_bc_operator_symmetric_and_natural(bc):
    L = 5
    n, N = (1 << L) + 1, ((1 << L) + 1) ** 2
    A = O.assemble(L, None, bc=bc)
    unk = _unknown_mask(L, bc)
    # symmetric: a_k[i] = a_{8-k}[i + off_k]
    for k in range(9):
        dy, dx = k // 3 - 1, k % 3 - 1
        for i in np.flatnonzero(unk)[::7]:
            iy, ix = divmod(i, n)
            jy, jx = iy + dy, ix + dx
            if 0 <= jx < n and 0 <= jy < n:
                assert A[k, i] == A[8 - k, jy * n + jx]
    # constants are in the kernel away from Dirichlet nodes: zero row sums on unknown rows
    # whose neighbours are all unknowns (natural boundary condition on the free sides)
    grid = unk.reshape(n, n)
    pad = np.pad(grid, 1, constant_values=True)
    ok = np.ones_like(grid)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ok &= pad[1 + dy:1 + dy + n, 1 + dx:1 + dx + n]
    rows = np.flatnonzero(ok.ravel() & unk)
    assert len(rows) > 0
    assert np.max(np.abs(A[:, rows].sum(axis=0))) <= 1e-14
    # Dirichlet rows are identity rows
    d = np.flatnonzero(~unk)
    assert np.all(A[4, d] == 1.0) and np.all(A[[0, 1, 2, 3, 5, 6, 7, 8]][:, d] == 0.0)


def test_mixed_bc_free_side_stencil_closed_form():
    # a = 1: an interior node of a free side keeps half the interior stencil 8/3, -1/3:
    # diagonal 4/3, along the side -1/6, into the domain -1/3 (edge and both corners)
    L = 4
    n, N = (1 << L) + 1, ((1 << L) + 1) ** 2
    A = O.assemble(L, None, bc=LR)
    i = 0 * n + 5                        # bottom side (y = 0), ix = 5
    expect = {4: 4 / 3, 3: -1 / 6, 5: -1 / 6, 7: -1 / 3, 6: -1 / 3, 8: -1 / 3, 0: 0.0, 1: 0.0, 2: 0.0}
    for k, v in expect.items():
        assert abs(A[k, i] - v) <= 4e-16, (k, A[k, i], v)


def test_mixed_bc_transfers_adjoint_and_exact():
    Lf = 5
    nf, nc = (1 << Lf) + 1, (1 << (Lf - 1)) + 1
    rng = np.random.default_rng(11)
    r = rng.uniform(-1, 1, nf * nf) * _unknown_mask(Lf, LR)
    e = rng.uniform(-1, 1, nc * nc) * _unknown_mask(Lf - 1, LR)
    Rr = O.restrict(Lf, r, bc=LR)
    Pe = O.prolong_add(Lf, e, np.zeros(nf * nf), bc=LR)
    assert abs(np.dot(Rr, e) - np.dot(r, Pe)) <= 1e-12 * np.sum(np.abs(Rr * e))
    # P reproduces g(x) (alpha + beta y) for g piecewise linear on the coarse grid, zero at
    # x = 0, 1: exact on every unknown node, including the free sides y = 0, 1
    g = rng.uniform(-1, 1, nc)
    g[0] = g[-1] = 0.0
    Yc = np.arange(nc) / (nc - 1)
    ec = (g[None, :] * (0.3 + 0.7 * Yc[:, None])).ravel()
    gf = np.interp(np.arange(nf) / 2.0, np.arange(nc), g)
    Yf = np.arange(nf) / (nf - 1)
    expect = (gf[None, :] * (0.3 + 0.7 * Yf[:, None])).ravel()
    got = O.prolong_add(Lf, ec, np.zeros(nf * nf), bc=LR)
    assert np.max(np.abs(got - expect)) <= 1e-15


def test_mixed_bc_coarse_solve_exact():
    L = 3
    A = O.assemble(L, None, bc=LR)
    unk = _unknown_mask(L, LR)
    b = np.random.default_rng(5).uniform(-1, 1, unk.size) * unk
    x = O.coarse_solve(L, A, b, bc=LR)
    r = O.defect(L, A, b, x)
    assert np.max(np.abs(r)) <= 1e-13 and np.all(x[~unk] == 0.0)


def test_mixed_bc_manufactured_solution_second_order():
    # u = sin(pi x) cos(pi y): zero at x = 0, 1, zero normal derivative at y = 0, 1
    errs = []
    for L in range(3, 8):
        b = O.load_sincos(L)
        x, st = O.mg_solve(L, b, tol=1e-11, bc=LR)
        assert st["converged"]
        errs.append(O.l2_error_sincos(L, x))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.7 < q < 4.3 for q in ratios[1:]), ratios
    assert errs[-1] < 2e-4


def test_boundary_mask_needs_a_dirichlet_side():
    with pytest.raises(ValueError):
        O.assemble(3, None, bc=0)


# ------------------------------------------ CG coarse solver and CG with a multigrid preconditioner
@pytest.mark.parametrize("Lc,bc", [(2, 15), (3, 15), (4, 15), (3, LR), (4, 1)])
def test_coarse_cg_matches_cholesky(Lc, bc):
    coef = I.lognormal_coef(Lc, 70 + Lc)
    A = O.assemble(Lc, coef, bc=bc)
    b = np.random.default_rng(Lc).uniform(-1, 1, A.shape[1]) * _unknown_mask(Lc, bc)
    x_cg, steps = O.coarse_solve(Lc, A, b, bc=bc, cg=True, steps=True)
    x_ex = O.coarse_solve(Lc, A, b, bc=bc)
    assert 0 < steps <= 2 * int(_unknown_mask(Lc, bc).sum()) + 10
    assert np.max(np.abs(x_cg - x_ex)) <= 1e-11 * np.max(np.abs(x_ex))
    assert np.max(np.abs(O.defect(Lc, A, b, x_cg))) <= 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("Lc,bc", [(2, 15), (3, 15), (3, LR)])
def test_coarse_cg_finite_termination(Lc, bc):
    # exact-arithmetic CG ends after as many steps as the matrix has distinct eigenvalues whose
    # eigenvectors the right-hand side excites; a = 1 has many repeated eigenvalues
    A = O.assemble(Lc, None, bc=bc)
    n = (1 << Lc) + 1
    unk = np.flatnonzero(_unknown_mask(Lc, bc))
    M = np.zeros((len(unk), len(unk)))
    pos = {g: i for i, g in enumerate(unk)}
    for i, g in enumerate(unk):
        iy, ix = divmod(g, n)
        for k in range(9):
            jy, jx = iy + k // 3 - 1, ix + k % 3 - 1
            if 0 <= jx < n and 0 <= jy < n and jy * n + jx in pos:
                M[i, pos[jy * n + jx]] = A[k, g]
    ev = np.linalg.eigvalsh(M)
    distinct = 1 + int(np.sum(np.diff(np.sort(ev)) > 1e-9 * ev.max()))
    b = np.zeros(A.shape[1])
    b[unk] = np.random.default_rng(3).uniform(-1, 1, len(unk))
    _, steps = O.coarse_solve(Lc, A, b, bc=bc, cg=True, steps=True)
    assert steps <= distinct + 1, (steps, distinct)


def test_mg_with_coarse_cg_follows_the_exact_coarse_solve():
    L = 7
    coef = I.lognormal_coef(L, 5)
    b = I.rhs_uniform(L, 6)
    for coarse_L in (2, 3):
        x1, s1 = O.mg_solve(L, b, coef=coef, coarse_L=coarse_L)
        x2, s2 = O.mg_solve(L, b, coef=coef, coarse_L=coarse_L, coarse_cg=True)
        assert s1["cycles"] == s2["cycles"] and s2["converged"]
        assert np.max(np.abs(x1 - x2)) <= 1e-9 * np.max(np.abs(x1))


@pytest.mark.parametrize("bc,coarse_cg", [(15, False), (15, True), (LR, False)])
def test_preconditioner_is_symmetric(bc, coarse_cg):
    # V(nu, nu) with damped Jacobi and R = P^T is an A-self-adjoint error propagation, so
    # M = (I - E) A^-1 is symmetric: <M u, v> = <u, M v>
    L = 5
    coef = I.lognormal_coef(L, 8)
    rng = np.random.default_rng(9)
    unk = _unknown_mask(L, bc)
    u = rng.uniform(-1, 1, unk.size) * unk
    v = rng.uniform(-1, 1, unk.size) * unk
    Mu = O.precondition(L, u, coef=coef, bc=bc, coarse_cg=coarse_cg)
    Mv = O.precondition(L, v, coef=coef, bc=bc, coarse_cg=coarse_cg)
    a, b = np.dot(Mu, v), np.dot(u, Mv)
    assert abs(a - b) <= 1e-11 * np.sum(np.abs(Mu * v))
    assert np.dot(Mu, u) > 0 and np.dot(Mv, v) > 0                 # and positive definite


@pytest.mark.parametrize("L,prec", [(5, 0), (6, 0), (5, 1)])
def test_pcg_follows_scipy_cg(L, prec):
    # the same iteration run by scipy's conjugate gradient with the oracle's operator and
    # preconditioner as linear operators
    spla = pytest.importorskip("scipy.sparse.linalg")
    coef = I.lognormal_coef(L, 30 + L)
    b = I.rhs_uniform(L, 31)
    A = O.assemble(L, coef)
    N = b.size
    Aop = spla.LinearOperator((N, N), matvec=lambda v: O.spmv(L, A, v), dtype=np.float64)
    Mop = spla.LinearOperator((N, N), matvec=lambda v: O.precondition(L, v, coef=coef, prec=prec),
                              dtype=np.float64)
    k = 5
    xs, info = spla.cg(Aop, b, rtol=0.0, atol=0.0, maxiter=k, M=Mop)
    xo, st = O.pcg_solve(L, b, coef=coef, prec=prec, tol=0.0, max_iters=k)
    assert info == k and st["outer_iters"] == k and st["cycles"] == k
    assert np.linalg.norm(xo - xs) <= 1e-10 * np.linalg.norm(xs)


def test_pcg_with_exact_preconditioner_takes_one_step():
    # coarse_L = L: the "cycle" is the exact solve, M = A^-1, so p_0 = A^-1 b and alpha = 1
    L = 3
    coef = I.lognormal_coef(L, 4)
    b = I.rhs_uniform(L, 5)
    x, st = O.pcg_solve(L, b, coef=coef, coarse_L=L, tol=1e-12)
    assert st["outer_iters"] == 1 and st["relres"] <= 1e-14


def test_pcg_accelerates_multigrid():
    L = 7
    coef = I.lognormal_coef(L, 12)
    b = I.rhs_uniform(L, 13)
    _, sm = O.mg_solve(L, b, coef=coef)
    x64, s64, h = O.pcg_solve(L, b, coef=coef, history=True)
    assert s64["converged"] and s64["relres"] <= 1.0001e-8
    assert s64["outer_iters"] < sm["cycles"]
    assert np.all(np.diff(h) < 0)                                  # residual falls every step
    for prec in (1, 2):
        x, s = O.pcg_solve(L, b, coef=coef, prec=prec)
        assert s["converged"] and s["relres"] <= 1.0001e-8
        assert abs(s["outer_iters"] - s64["outer_iters"]) <= 1
        assert np.linalg.norm(x - x64) <= 1e-7 * np.linalg.norm(x64)


def test_pcg_mixed_boundaries_manufactured_solution():
    L = 6
    b = O.load_sincos(L)
    xm, _ = O.mg_solve(L, b, bc=LR, tol=1e-11)
    xp, sp = O.pcg_solve(L, b, bc=LR, tol=1e-11)
    assert sp["converged"]
    assert abs(O.l2_error_sincos(L, xp) / O.l2_error_sincos(L, xm) - 1) < 1e-6


# ------------------------------------------- four-band matrices and the shallow-water prediction step
def _dense_band4(offsets, bands, n):
    """The matrix itself, entry by entry: M[i, i + off_k] = band_k[i] where the column exists."""
    M = np.zeros((n, n))
    for k, d in enumerate(offsets):
        for i in range(n):
            if 0 <= i + d < n:
                M[i, i + d] += bands[k][i]
    return M


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_swe_predict_exact_on_integers(dtype):
    # small integers: every product and sum is exact in both precisions, so the result must equal
    # the integer linear combination exactly (pins indexing, offsets, edges and the operands)
    n = 61
    rng = np.random.default_rng(1)
    offs = np.array([[-2, -1, 1, 2], [-12, -6, 6, 12], [-1, 0, 1, 3], [-70, 4, 7, 60]])
    bands = rng.integers(-3, 4, (4, 4, n))
    u, v, w, s = (rng.integers(-5, 6, n) for _ in range(4))
    ref = u + s
    for m, x in enumerate((v, w, u, u)):
        ref = ref + _dense_band4(offs[m], bands[m], n).astype(np.int64) @ x
    got = O.swe_predict(offs, bands.astype(dtype), u.astype(dtype), v.astype(dtype), w.astype(dtype),
                        s.astype(dtype))
    assert got.dtype == dtype
    np.testing.assert_array_equal(got.astype(np.int64), ref)
    got = O.swe_predict(offs, bands.astype(dtype), u.astype(dtype), v.astype(dtype), w.astype(dtype))
    np.testing.assert_array_equal(got.astype(np.int64), ref - s)


def test_band4_against_scipy_diagonals():
    sp = pytest.importorskip("scipy.sparse")
    n = 300
    rng = np.random.default_rng(2)
    offs = [-17, -1, 2, 17]
    bands = rng.uniform(-1, 1, (4, n))
    x = rng.uniform(-1, 1, n)
    diags = [bands[k][max(0, -d):n - max(0, d)] for k, d in enumerate(offs)]
    M = sp.diags(diags, offs, shape=(n, n))
    y = O.band4_spmv(offs, bands, x)
    ref = M @ x
    assert np.max(np.abs(y - ref)) <= 1e-15 * 4 * np.max(np.abs(bands)) * np.max(np.abs(x))
    y32 = O.band4_spmv(offs, bands.astype(np.float32), x.astype(np.float32))
    assert np.max(np.abs(y32 - ref)) <= 4 * 4 * 2.0 ** -24 * 4


def test_band4_degenerate_sizes():
    offs = [[5, 6, 7, 8]] * 4                  # every column beyond n = 4: no entries
    bands = np.ones((4, 4, 4))
    u = np.arange(4.0)
    np.testing.assert_array_equal(O.swe_predict(offs, bands, u, u, u, u), 2 * u)
    assert O.swe_predict(offs, np.ones((4, 4, 0)), np.zeros(0), np.zeros(0), np.zeros(0)).size == 0
