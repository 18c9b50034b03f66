"""BLAS level-1 kernels (include/hn_blas1.h) against the oracle (Sec. 6.1 measures axpy on every
backend).  axpy rounds once per element, as the oracle does, so it must match bit for bit; dot and
nrm2 sum in a fixed order and are compared with the exactly summed oracle within that order's
rounding bound; two calls must give identical bits."""
import ctypes

import numpy as np
import pytest

import oracle as O
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu
SIZES = [0, 1, 3, 17, 1000, 16384, 16385, 100003, (1 << 22) + 7]


@pytest.fixture(scope="module")
def hn():
    return require_gpu()


def _data(n, dtype, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, n).astype(dtype), rng.uniform(-1, 1, n).astype(dtype)


def _dot_tol(dtype, x, y):
    s = float(np.sum(np.abs(x.astype(np.float64) * y.astype(np.float64))))
    m = max(1, -(-len(x) // 16384))
    if dtype == np.float32:                  # FP32 chains of <= 16 products, the rest in FP64
        return 17 * 2.0 ** -24 * s + (40 + m) * 2.0 ** -53 * s
    return (16 + 40 + m) * 2.0 ** -53 * s


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("offset", [0, 1])
def test_axpy_bit_exact(hn, dtype, n, offset):
    import torch
    x, y = _data(n + offset, dtype, 10 + n)
    xt, yt = torch.from_numpy(x).cuda()[offset:], torch.from_numpy(y).cuda()[offset:]   # offset 1: unaligned
    hn.hn_axpy(-0.37, xt, yt)
    ref = O.axpy(-0.37, x[offset:], y[offset:])
    np.testing.assert_array_equal(yt.cpu().numpy(), ref)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", SIZES)
def test_dot_nrm2_within_bound_and_deterministic(hn, dtype, n):
    import torch
    x, y = _data(n, dtype, 20 + n)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    r = torch.zeros(4, dtype=torch.float64, device="cuda")
    hn.hn_dot(xt, yt, r[0:])
    hn.hn_dot(xt, yt, r[1:])
    hn.hn_nrm2(xt, r[2:])
    got = r.cpu().numpy()
    ref = O.dot(x, y)
    assert abs(got[0] - ref) <= _dot_tol(dtype, x, y)
    assert got[0] == got[1]                   # same bits every call
    ref2 = np.sqrt(O.dot(x, x))
    tol2 = 0.5 * _dot_tol(dtype, x, x) / max(ref2, 1e-300) + 2 * 2.0 ** -53 * ref2
    assert abs(got[2] - ref2) <= tol2


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_dot_order_does_not_depend_on_alignment(hn, dtype):
    # unaligned vectors take the element-by-element path in the same order as the 16-byte loads
    import torch
    n = 100003
    x, y = _data(n + 1, dtype, 31)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    r = torch.zeros(2, dtype=torch.float64, device="cuda")
    hn.hn_dot(xt[1:], yt[1:], r[0:])                      # 4 or 8 bytes off a 16-byte boundary
    hn.hn_dot(xt[1:].clone(), yt[1:].clone(), r[1:])      # aligned copies
    a, b = r.cpu().numpy()
    assert a == b


def test_blas1_rejects_bad_arguments(hn):
    L = hn.lib()
    assert L.hn_axpy(0, -1, 1.0, None, None, None) == hn.HN_ERR_ARG
    assert L.hn_axpy(7, 10, 1.0, None, None, None) == hn.HN_ERR_ARG
    assert L.hn_dot(0, 10, None, None, None, None) == hn.HN_ERR_ARG
    assert L.hn_nrm2(1, 5, None, None, None) == hn.HN_ERR_ARG
    assert L.hn_axpy(0, 0, 1.0, None, None, None) == hn.HN_OK      # n = 0: nothing to do
