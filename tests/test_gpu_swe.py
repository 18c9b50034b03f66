"""Four-band matrices at arbitrary band positions and the fused shallow-water prediction step
(Sec. 2.2, Sec. 4.1) on the GPU against the oracle, through the C ABI (hn_swe.h).

The rounding order is part of the operation's definition, so results are compared bit for bit,
on ragged lengths (not multiples of the 4-row thread group), windows that leave the vector at both
ends, offsets that are misaligned, zero, repeated or beyond +-n, and at the benchmark size."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_0904_4152_gb300 import hn
    return hn, torch


def _case(n, W, seed, dtype):
    rng = np.random.default_rng(seed)
    offs = np.array([[-2, -1, 1, 2], [-2 * W, -W, W, 2 * W], [-1, 0, 1, 2], [-W - 1, -W + 1, W - 1, W + 1]])
    bands = rng.uniform(-1, 1, (4, 4, n)).astype(dtype)
    u, v, w, s = (rng.uniform(-1, 1, n).astype(dtype) for _ in range(4))
    return offs, bands, u, v, w, s


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,W", [(1, 1), (3, 2), (4, 2), (7, 3), (129, 11), (1000, 31), (4099, 64)])
def test_swe_predict_bit_exact(env, dtype, n, W):
    hn, torch = env
    offs, bands, u, v, w, s = _case(n, W, n + W, dtype)
    db = [[_dev(torch, bands[m, k]) for k in range(4)] for m in range(4)]
    du, dv, dw, ds = (_dev(torch, a) for a in (u, v, w, s))
    out = torch.empty_like(du)
    for with_s in (True, False):
        hn.hn_swe_predict(offs, db, du, dv, dw, ds if with_s else None, out)
        ref = O.swe_predict(offs, bands, u, v, w, s if with_s else None)
        np.testing.assert_array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_band4_spmv_bit_exact_odd_offsets(env, dtype):
    hn, torch = env
    rng = np.random.default_rng(5)
    n = 2053
    for offs in ([-3, 0, 0, 5], [-2100, -7, 2053, 9], [6, -6, 1, -1], [-1, -2, -3, -5]):
        bands = rng.uniform(-1, 1, (4, n)).astype(dtype)
        x = rng.uniform(-1, 1, n).astype(dtype)
        y = torch.empty(n, dtype=torch.float32 if dtype == np.float32 else torch.float64, device="cuda")
        hn.hn_band4_spmv(offs, [_dev(torch, b) for b in bands], _dev(torch, x), y)
        np.testing.assert_array_equal(y.cpu().numpy(), O.band4_spmv(offs, bands, x))


def test_swe_predict_benchmark_size(env):
    # the size the benchmark times (a 4096 x 4096 grid, FP32), every entry
    hn, torch = env
    W = 4096
    n = W * W
    offs, bands, u, v, w, s = _case(n, W, 77, np.float32)
    db = [[_dev(torch, bands[m, k]) for k in range(4)] for m in range(4)]
    du, dv, dw, ds = (_dev(torch, a) for a in (u, v, w, s))
    out = torch.empty_like(du)
    hn.hn_swe_predict(offs, db, du, dv, dw, ds, out)
    np.testing.assert_array_equal(out.cpu().numpy(), O.swe_predict(offs, bands, u, v, w, s))


def test_swe_arguments_checked(env):
    hn, torch = env
    n = 64
    t = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    good = [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(4)]
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(hn.HnError) as e:                      # a band 4 bytes off alignment
        hn.hn_band4_spmv([0, 1, 2, 3], good[:3] + [t[1:]], x, x.clone())
    assert e.value.status == hn.HN_ERR_ARG
    with pytest.raises(ValueError):
        hn.hn_band4_spmv([0, 1, 2, 3], good, x, torch.zeros(n + 1, dtype=torch.float32, device="cuda"))
    empty = torch.zeros(0, dtype=torch.float32, device="cuda")
    hn.hn_band4_spmv([0, 1, 2, 3], [empty] * 4, empty, empty.clone())   # n = 0: nothing to do
