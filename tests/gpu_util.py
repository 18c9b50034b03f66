"""Helpers shared by the GPU tests: build/load the CUDA library, run solves through the C ABI,
and the oracle-side reference quantities."""
import numpy as np
import pytest

import oracle as O
from paper_0904_4152_gb300 import inputs as I


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_0904_4152_gb300 import hn
    return hn


def coef_levels(L, coef, coarse=2):
    """Oracle coefficient of every level (mean of the 4 children), {l: array or None}."""
    out = {L: coef}
    for l in range(L, coarse, -1):
        out[l - 1] = None if out[l] is None else O.coarsen_coef(l, out[l])
    return out


def solve(hn, L, b, coef=None, bc=O.ALL_DIRICHLET, **opts):
    A = hn.hn_band_create_bc(L, coef, bc)
    try:
        mg = hn.hn_mg_setup(A, **opts)
    finally:
        hn.hn_band_destroy(A)
    try:
        x, st, status = hn.hn_mg_solve(mg, L, b)
    finally:
        hn.hn_mg_destroy(mg)
    return x, st, status


def oracle_relres(L, coef, b, x, bc=O.ALL_DIRICHLET):
    A = O.assemble(L, coef, bc=bc)
    return np.linalg.norm(O.defect(L, A, b, x)) / np.linalg.norm(b)


def rand_interior(L, seed, dtype=np.float64):
    rng = np.random.default_rng(seed)
    n = (1 << L) + 1
    v = rng.uniform(-1, 1, n * n)
    v[~interior(L)] = 0.0
    return v.astype(dtype)


def rand_unknowns(L, bc, seed, dtype=np.float64):
    """U[-1,1] on the nodes off the Dirichlet sides of the side mask bc, 0 on them."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1, 1, ((1 << L) + 1) ** 2)
    v[~I.unknown_mask(L, bc)] = 0.0
    return v.astype(dtype)


def interior(L):
    n = (1 << L) + 1
    m = np.zeros((n, n), dtype=bool)
    m[1:-1, 1:-1] = True
    return m.ravel()


def abs_spmv(L, bands, x):
    """sum_k |a_k x_k| per row: the scale of the rounding error of a 9-term product."""
    return O.spmv(L, np.abs(bands), np.abs(x))
