"""The seeded input generators against their definitions: SplitMix64's published outputs, the
U[0,1) mapping, the right-hand-side and boundary recipes, the random-Fourier-feature field's
covariance, and the batch and arrival recipes.  CPU only."""
import numpy as np
import pytest

from paper_0904_4152_gb300 import inputs as I


def splitmix64_scalar(seed, count):
    # the generator as published: state += 0x9E3779B97F4A7C15, then the two xor-shift-multiply
    # rounds and a final xor-shift of the state
    mask = (1 << 64) - 1
    s, out = seed & mask, []
    for _ in range(count):
        s = (s + 0x9E3779B97F4A7C15) & mask
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_published_outputs():
    # reference outputs of SplitMix64 (Steele, Lea, Flood 2014) for seeds 0 and 1234567
    assert [int(v) for v in I.splitmix64(0, 4)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                    0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(v) for v in I.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]
    assert [int(v) for v in I.splitmix64(987654321, 64)] == splitmix64_scalar(987654321, 64)


def test_splitmix64_offsets_continue_the_stream():
    full = I.splitmix64(42, 100)
    np.testing.assert_array_equal(I.splitmix64(42, 30, start=70), full[70:])


def test_uniform01_uses_the_top_53_bits():
    raw = I.splitmix64(5, 1000)
    u = I.uniform01(5, 1000)
    assert u.min() >= 0.0 and u.max() < 1.0
    np.testing.assert_array_equal(u, np.array([float(int(v) >> 11) for v in raw]) * 2.0 ** -53)
    big = I.uniform01(6, 200_000)
    assert abs(big.mean() - 0.5) < 4 * np.sqrt(1 / 12 / big.size)
    assert abs(big.var() - 1 / 12) < 1e-3


@pytest.mark.parametrize("L", [2, 5])
def test_rhs_uniform_is_zero_on_the_boundary(L):
    n = (1 << L) + 1
    b = I.rhs_uniform(L, 3).reshape(n, n)
    assert not b[0].any() and not b[-1].any() and not b[:, 0].any() and not b[:, -1].any()
    inner = b[1:-1, 1:-1]
    assert inner.min() >= -1.0 and inner.max() < 1.0 and np.count_nonzero(inner) == inner.size
    np.testing.assert_array_equal(I.rhs_uniform(L, 3), b.ravel())
    assert not np.array_equal(I.rhs_uniform(L, 4), b.ravel())


@pytest.mark.parametrize("sides", [1, 5, 10, 15])
def test_rhs_with_a_side_mask_is_zero_exactly_on_the_dirichlet_sides(sides):
    L = 4
    n = (1 << L) + 1
    b = I.rhs_uniform_bc(L, 9, sides).reshape(n, n)
    rows = {1: b[0, :], 2: b[:, -1], 4: b[-1, :], 8: b[:, 0]}
    for bit, edge in rows.items():
        if sides & bit:
            assert not edge.any()
    free = I.unknown_mask(L, sides).reshape(n, n)
    assert np.count_nonzero(b[free]) == free.sum()
    if sides == 15:
        np.testing.assert_array_equal(free, I.interior_mask(L).reshape(n, n))


def test_gaussian_field_is_its_feature_sum():
    # the separable evaluation equals sqrt(2/M) sum_m cos(w_m . x + p_m) at the cell centres
    L, seed, ell, M = 3, 11, 0.1, 64
    g = I.gaussian_field(L, seed, ell, features=M).reshape(1 << L, 1 << L)
    u = I.uniform01(seed, 3 * M)
    r = np.sqrt(-2.0 * np.log(1.0 - u[:M]))
    w = np.stack([r * np.cos(2 * np.pi * u[M:2 * M]), r * np.sin(2 * np.pi * u[M:2 * M])], 1) / ell
    p = 2 * np.pi * u[2 * M:]
    for ey, ex in [(0, 0), (2, 5), (7, 7), (6, 1)]:
        x = np.array([(ex + 0.5) / 8, (ey + 0.5) / 8])
        direct = np.sqrt(2.0 / M) * np.cos(w @ x + p).sum()
        assert abs(g[ey, ex] - direct) < 1e-10


def test_gaussian_field_covariance_is_squared_exponential():
    # over many seeds E[g(x) g(x')] = exp(-|x - x'|^2 / (2 ell^2)); pairs along x at distances 0,
    # 0.125 (2 cells: e^-0.78) and 0.3125 (5 cells: ~0) from cell (8, 3)
    L, ell, seeds = 4, 0.1, 400
    nc = 1 << L
    fields = np.array([I.gaussian_field(L, s, ell).reshape(nc, nc) for s in range(seeds)])
    h = 1.0 / nc
    for dx_cells in (0, 2, 5):
        d = dx_cells * h
        cov = np.mean(fields[:, 8, 3] * fields[:, 8, 3 + dx_cells])
        assert abs(cov - np.exp(-d * d / (2 * ell * ell))) < 0.2
    assert abs(fields.mean()) < 0.05


def test_lognormal_coefficients_are_positive_and_seeded():
    a = I.lognormal_coef(5, 1000)
    assert a.shape == (32 * 32,) and (a > 0).all()
    np.testing.assert_array_equal(a, np.exp(I.gaussian_field(5, 1000)))
    c, b = I.batch_problem(3, 5)
    np.testing.assert_array_equal(c, I.lognormal_coef(5, 1003))
    np.testing.assert_array_equal(b, I.rhs_uniform(5, 2003))


def test_batch_levels_cover_five_to_nine():
    lv = I.batch_levels(256, seed=0)
    assert lv.min() == 5 and lv.max() == 9 and set(lv.tolist()) == {5, 6, 7, 8, 9}
    np.testing.assert_array_equal(lv, I.batch_levels(256, seed=0))


def test_serve_arrivals_are_poisson_with_uniform_levels():
    count, rate = 30_000, 250.0
    arrivals, levels, seeds = I.serve_requests(count, rate, seed=7)
    gaps = np.diff(np.concatenate([[0.0], arrivals]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() * rate - 1.0) < 0.03             # exponential gaps of mean 1/rate
    assert abs(gaps.std() * rate - 1.0) < 0.05              # (standard deviation = mean)
    share = np.bincount(levels - 6, minlength=6) / count
    assert levels.min() == 6 and levels.max() == 11 and np.abs(share - 1 / 6).max() < 0.015
    np.testing.assert_array_equal(seeds, np.arange(count) + 10_000)
