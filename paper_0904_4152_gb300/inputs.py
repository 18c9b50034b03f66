"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the CPU oracle.

This module holds no solver arithmetic: it only draws numbers.  Every value comes from the
SplitMix64 generator (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), whose output k (k = 0, 1, ...) for a seed s is mix(s + (k+1) * 0x9E3779B97F4A7C15);
U[0,1) uses the top 53 bits.  Workload recipes:

* right-hand sides: U[-1, 1] on interior nodes, 0 on the Dirichlet boundary; with a side mask
  (bit 1 y = 0, 2 x = 1, 4 y = 1, 8 x = 0 Dirichlet), U[-1, 1] on every node off the Dirichlet
  sides, including the free Neumann sides;
* coefficient fields: a = exp(sigma * g) per cell, g a smooth Gaussian field with
  squared-exponential covariance (correlation length ell) sampled by M random Fourier features,
  g(x) = sqrt(2/M) sum_m cos(w_m . x + p_m), w_m ~ N(0, ell^-2 I), p_m ~ U[0, 2 pi), evaluated at
  the cell centres (the field is a function of x, the same at every refinement level);
* batches: problem j has L_j ~ U{5..9}, field seed 1000 + j, right-hand side seed 2000 + j;
* serving: Poisson arrivals (exponential gaps), L uniform over {6..11}, per-request seeds.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 seeded with ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def n_of(L: int) -> int:
    return (1 << L) + 1


def interior_mask(L: int) -> np.ndarray:
    n = n_of(L)
    m = np.zeros((n, n), dtype=bool)
    m[1:-1, 1:-1] = True
    return m.ravel()


def rhs_uniform(L: int, seed: int) -> np.ndarray:
    """Discrete right-hand side b: U[-1,1] on interior nodes, 0 on the boundary."""
    n = n_of(L)
    b = np.zeros(n * n)
    m = interior_mask(L)
    b[m] = uniform01(seed, int(m.sum())) * 2.0 - 1.0
    return b


def unknown_mask(L: int, dirichlet_sides: int) -> np.ndarray:
    """Nodes that are not on a Dirichlet side of the side mask."""
    n = n_of(L)
    m = np.ones((n, n), dtype=bool)
    if dirichlet_sides & 1: m[0, :] = False
    if dirichlet_sides & 2: m[:, -1] = False
    if dirichlet_sides & 4: m[-1, :] = False
    if dirichlet_sides & 8: m[:, 0] = False
    return m.ravel()


def rhs_uniform_bc(L: int, seed: int, dirichlet_sides: int) -> np.ndarray:
    """Right-hand side U[-1,1] on the unknowns of a side mask, 0 on its Dirichlet sides."""
    n = n_of(L)
    b = np.zeros(n * n)
    m = unknown_mask(L, dirichlet_sides)
    b[m] = uniform01(seed, int(m.sum())) * 2.0 - 1.0
    return b


def gaussian_field(L: int, seed: int, ell: float = 0.1, features: int = 512) -> np.ndarray:
    """Smooth unit-variance Gaussian field at the (2^L)^2 cell centres, row-major (ey, ex)."""
    u = uniform01(seed, 3 * features)
    u1, u2, u3 = u[:features], u[features:2 * features], u[2 * features:]
    r = np.sqrt(-2.0 * np.log1p(-u1))          # Box-Muller: two independent normals
    wx = r * np.cos(2 * np.pi * u2) / ell
    wy = r * np.sin(2 * np.pi * u2) / ell
    ph = 2 * np.pi * u3
    nc = 1 << L
    c = (np.arange(nc) + 0.5) / nc              # cell-centre coordinates
    # cos(wx x + wy y + p) = cos(wx x + p) cos(wy y) - sin(wx x + p) sin(wy y)
    ax = np.outer(wx, c) + ph[:, None]          # (M, nc) over x
    ay = np.outer(wy, c)                        # (M, nc) over y
    g = np.cos(ay).T @ np.cos(ax) - np.sin(ay).T @ np.sin(ax)   # [ey, ex]
    return (np.sqrt(2.0 / features) * g).ravel()


def lognormal_coef(L: int, seed: int, sigma: float = 1.0, ell: float = 0.1) -> np.ndarray:
    """Per-cell coefficient a = exp(sigma * g)."""
    return np.exp(sigma * gaussian_field(L, seed, ell))


def batch_levels(count: int = 256, seed: int = 0, lo: int = 5, hi: int = 9) -> np.ndarray:
    """Refinement levels L_j ~ U{lo..hi}."""
    return (np.floor(uniform01(seed, count) * (hi - lo + 1)).astype(np.int64) + lo)


def batch_problem(j: int, L: int):
    """Coefficient field and right-hand side of problem j of a batch."""
    return lognormal_coef(L, 1000 + j), rhs_uniform(L, 2000 + j)


def serve_requests(count: int, rate_per_s: float, seed: int = 7, lo: int = 6, hi: int = 11):
    """Arrival times (s, Poisson process), levels uniform over {lo..hi}, per-request seeds."""
    u = uniform01(seed, 2 * count)
    gaps = -np.log1p(-u[:count]) / rate_per_s
    arrivals = np.cumsum(gaps)
    levels = np.floor(u[count:] * (hi - lo + 1)).astype(np.int64) + lo
    seeds = np.arange(count, dtype=np.int64) + 10_000
    return arrivals, levels, seeds
