"""End-to-end parity of the GPU multigrid solves with the oracle, through the C ABI.

Gates (the method iterates, so two independently stopped solves differ by about the tolerance):
  G1  FP64 V cycles in lockstep with the oracle (same cycle count): ||dx|| / ||x|| <= 1e-9.
  G2  every GPU result, checked with the oracle's FP64 operator: ||b - A x|| / ||b|| <= 1e-8.
  G3  mixed-precision results against the oracle solved to 1e-13: <= 1e-9 when the GPU side is
      also run to a tighter stop (1e-11)."""
import numpy as np
import pytest

import oracle as O
from paper_0904_4152_gb300 import inputs as I
from gpu_util import oracle_relres, require_gpu, solve

pytestmark = pytest.mark.gpu
RELRES = 1.0001e-8


@pytest.fixture(scope="module")
def hn():
    return require_gpu()


@pytest.mark.parametrize("L,lognormal", [(3, False), (6, False), (6, True), (9, True)])
def test_g1_fp64_lockstep(hn, L, lognormal):
    coef = I.lognormal_coef(L, 300 + L) if lognormal else None
    b = I.rhs_uniform(L, 301)
    k = 4
    x, st, status = solve(hn, L, b, coef, tol=0.0, max_cycles=k)
    assert status == hn.HN_ERR_NOT_CONVERGED and st["cycles"] == k
    xr, sr = O.mg_solve(L, b, coef=coef, tol=0.0, max_cycles=k)
    assert sr["cycles"] == k
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-9
    assert abs(st["relres"] - sr["relres"]) <= 1e-6 * sr["relres"]


def test_g2_config_small_sinsin(hn):
    # L=6, a=1, f = 2 pi^2 sin(pi x) sin(pi y), V(2,2), omega 0.7, coarse L=2, tol 1e-8
    L = 6
    b = O.load_sinsin(L)
    x, st, status = solve(hn, L, b)
    xr, sr = O.mg_solve(L, b)
    assert status == hn.HN_OK and st["relres"] <= 1e-8
    assert oracle_relres(L, None, b, x) <= RELRES
    assert st["cycles"] == sr["cycles"]
    e_gpu, e_or = O.l2_error_sinsin(L, x), O.l2_error_sinsin(L, xr)
    assert abs(e_gpu / e_or - 1) < 1e-6


@pytest.mark.parametrize("prec", [1, 2])
def test_g2_g3_mixed_precision(hn, prec):
    L = 7
    coef = I.lognormal_coef(L, 0)
    b = I.rhs_uniform(L, 1)
    x, st, status = solve(hn, L, b, coef, prec=prec)
    assert status == hn.HN_OK
    assert oracle_relres(L, coef, b, x) <= RELRES
    assert st["outer_iters"] >= 2 and st["inner_cycles"] >= st["outer_iters"]
    xs, _ = O.mg_solve(L, b, coef=coef, tol=1e-13)
    # the oracle's own DC takes the same number of outer steps (+-1)
    _, so = O.mg_solve(L, b, coef=coef, prec=prec)
    assert abs(so["outer_iters"] - st["outer_iters"]) <= 1
    x2, st2, status2 = solve(hn, L, b, coef, prec=prec, tol=1e-11)
    assert status2 == hn.HN_OK
    assert np.linalg.norm(x2 - xs) / np.linalg.norm(xs) <= 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_g2_config_L10(hn, prec):
    # L=10 (1025^2 nodes), a=1, b ~ U[-1,1] seed 0: FP64 MG and FP32-inner defect correction
    L = 10
    b = I.rhs_uniform(L, 0)
    x, st, status = solve(hn, L, b, prec=prec)
    assert status == hn.HN_OK
    assert oracle_relres(L, None, b, x) <= RELRES


def test_device_and_host_pointers_agree(hn):
    torch = pytest.importorskip("torch")
    L = 7
    b = I.rhs_uniform(L, 9)
    A = hn.hn_band_create(L)
    mg = hn.hn_mg_setup(A, prec=1)
    hn.hn_band_destroy(A)
    try:
        xh, _, _ = hn.hn_mg_solve(mg, L, b)
        bd = torch.from_numpy(b).cuda()
        xd, _, _ = hn.hn_mg_solve(mg, L, bd)
        np.testing.assert_array_equal(xd.cpu().numpy(), xh)
        # a converged initial guess: no cycle is needed
        x0 = xh.copy()
        x1, st, status = hn.hn_mg_solve(mg, L, b, x=x0, x_is_guess=True)
        assert status == hn.HN_OK and st["cycles"] == 0
    finally:
        hn.hn_mg_destroy(mg)


def test_fp64_converged_guess_and_zero_rhs(hn):
    L = 5
    b = I.rhs_uniform(L, 3)
    A = hn.hn_band_create(L)
    mg = hn.hn_mg_setup(A)
    hn.hn_band_destroy(A)
    try:
        x, st, _ = hn.hn_mg_solve(mg, L, b)
        x1, st1, status = hn.hn_mg_solve(mg, L, b, x=x.copy(), x_is_guess=True)
        assert status == hn.HN_OK and st1["cycles"] == 0
        np.testing.assert_array_equal(x1, x)
        z, stz, status = hn.hn_mg_solve(mg, L, np.zeros_like(b), x=np.ones_like(b), x_is_guess=True)
        assert status == hn.HN_OK and np.all(z == 0) and stz["cycles"] == 0
    finally:
        hn.hn_mg_destroy(mg)


def test_invalid_inputs_fail_cleanly(hn):
    L = 4
    A = hn.hn_band_create(L)
    mg = hn.hn_mg_setup(A, prec=1)
    hn.hn_band_destroy(A)
    try:
        b = I.rhs_uniform(L, 1)
        bad = b.copy()
        bad[3] = 1.0                                    # boundary node
        with pytest.raises(hn.HnError) as e:
            hn.hn_mg_solve(mg, L, bad)
        assert e.value.status == hn.HN_ERR_ARG
        nan = b.copy()
        nan[40] = np.nan
        with pytest.raises(hn.HnError) as e:
            hn.hn_mg_solve(mg, L, nan)
        assert e.value.status == hn.HN_ERR_NONFINITE
        x, st, status = hn.hn_mg_solve(mg, L, b)          # the handle still works
        assert status == hn.HN_OK
    finally:
        hn.hn_mg_destroy(mg)
    A = hn.hn_band_create(L)
    mg = hn.hn_mg_setup(A, max_cycles=2, tol=1e-14)
    hn.hn_band_destroy(A)
    try:
        x, st, status = hn.hn_mg_solve(mg, L, I.rhs_uniform(L, 1))
        assert status == hn.HN_ERR_NOT_CONVERGED and st["cycles"] == 2
    finally:
        hn.hn_mg_destroy(mg)
    A = hn.hn_band_create(L)
    try:
        for bad in (dict(pre=0), dict(pre=2, post=1), dict(omega=2.5), dict(coarse_L=5),
                    dict(inner_tol=1.5)):
            with pytest.raises(hn.HnError) as e:
                hn.hn_mg_setup(A, **bad)
            assert e.value.status == hn.HN_ERR_ARG
    finally:
        hn.hn_band_destroy(A)


@pytest.mark.parametrize("L", [2, 3])
def test_degenerate_levels(hn, L):
    # L = coarse level: the exact coarse solve is the whole cycle
    b = I.rhs_uniform(L, 4)
    for prec in (0, 1, 2):
        x, st, status = solve(hn, L, b, prec=prec)
        assert status == hn.HN_OK and oracle_relres(L, None, b, x) <= RELRES


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_alone_equals_in_mix(hn, prec):
    levels = [2, 5, 7, 3, 6, 8, 5]
    mgs, bs, coefs = [], [], []
    for j, L in enumerate(levels):
        coef, b = I.batch_problem(j, L)
        A = hn.hn_band_create(L, coef)
        mgs.append(hn.hn_mg_setup(A, prec=prec))
        hn.hn_band_destroy(A)
        bs.append(b)
        coefs.append(coef)
    try:
        xs, stats, status = hn.hn_mg_solve_batch(mgs, levels, bs)
        assert status == hn.HN_OK
        for j, L in enumerate(levels):
            xa, sa, _ = hn.hn_mg_solve(mgs[j], L, bs[j])
            np.testing.assert_array_equal(xs[j], xa)              # bit-identical alone / in mix
            assert stats[j]["cycles"] == sa["cycles"]
            assert oracle_relres(L, coefs[j], bs[j], xs[j]) <= RELRES
        xs2, _, _ = hn.hn_mg_solve_batch(mgs, levels, bs)        # cached engine, same result
        for a, c in zip(xs, xs2):
            np.testing.assert_array_equal(a, c)
    finally:
        for m in mgs:
            hn.hn_mg_destroy(m)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_in_the_persistent_kernels_gives_the_same_bits(hn, prec):
    # levels 5..9 in the two persistent kernels of each cycle (tail level 4): the work-list path,
    # the lagged checks of up to two problems per level in the last block to reach the barrier
    # (levels 5, 8) and of more problems spread over the blocks (levels 6, 7)
    levels = [5, 7, 6, 8, 7, 6, 5, 8, 9, 6, 7]
    mgs, bs = [], []
    for j, L in enumerate(levels):
        coef, b = I.batch_problem(80 + j, L)
        A = hn.hn_band_create(L, coef)
        mgs.append(hn.hn_mg_setup(A, prec=prec))
        hn.hn_band_destroy(A)
        bs.append(b)
    try:
        ref, sref, status = hn.hn_mg_solve_batch(mgs, levels, bs)
        assert status == hn.HN_OK
        for m in mgs:
            hn.hn_mg_set_tuning(m, 4, 1, 2, 0, 1, 0, 10)
        xs, stats, status = hn.hn_mg_solve_batch(mgs, levels, bs)
        assert status == hn.HN_OK
        for j in range(len(levels)):
            np.testing.assert_array_equal(xs[j], ref[j])
            assert stats[j]["cycles"] == sref[j]["cycles"]
        xa, sa, _ = hn.hn_mg_solve(mgs[8], levels[8], bs[8])     # alone, same shape
        np.testing.assert_array_equal(xa, ref[8])
    finally:
        for m in mgs:
            hn.hn_mg_destroy(m)


def test_fp16_large_level_alone_equals_in_batch(hn):
    # alone, an engine of one problem passes its descriptors by value (and at L = 10 its levels
    # take the bulk-sized grids); in a batch the same kernels walk the work lists: same bits
    levels = [10, 6]
    mgs, bs = [], []
    for j, L in enumerate(levels):
        coef, b = I.batch_problem(70 + j, L)
        A = hn.hn_band_create(L, coef)
        mgs.append(hn.hn_mg_setup(A, prec=2))
        hn.hn_band_destroy(A)
        bs.append(b)
    try:
        xs, stats, status = hn.hn_mg_solve_batch(mgs, levels, bs)
        assert status == hn.HN_OK
        xa, sa, _ = hn.hn_mg_solve(mgs[0], levels[0], bs[0])
        np.testing.assert_array_equal(xs[0], xa)
        assert stats[0]["cycles"] == sa["cycles"]
    finally:
        for m in mgs:
            hn.hn_mg_destroy(m)


@pytest.mark.parametrize("slots", [4, 1])
def test_server_results_match_alone(hn, slots):
    # one slot: the engine of one problem passes descriptors by value and recaptures its graphs
    # whenever the member changes
    srv = hn.hn_server_create(2 << 30, slots)
    try:
        reqs = []
        for j, L in enumerate([6, 8, 5, 7, 6, 9, 4]):
            coef, b = I.batch_problem(j, L)
            t = hn.hn_mg_submit(srv, L, b, coef, prec=1)
            reqs.append((t, L, coef, b))
        for t, L, coef, b in reqs:
            status, x, st = hn.hn_mg_poll(srv, t, L, timeout_ns=60_000_000_000)
            assert status == hn.HN_OK
            xa, sa, _ = solve(hn, L, b, coef, prec=1)
            np.testing.assert_array_equal(x, xa)
            assert st["cycles"] == sa["cycles"]
        info = hn.hn_server_query(srv)
        assert info["completed"] == len(reqs) and info["active"] == 0
        status, _, _ = hn.hn_mg_poll(srv, reqs[0][0], 6, timeout_ns=0)   # forgotten ticket
    except hn.HnError as e:
        assert e.status == hn.HN_ERR_ARG
    finally:
        hn.hn_server_destroy(srv)


@pytest.mark.parametrize("slots", [4, 1])
def test_server_lanes_of_small_and_large_requests_match_alone(hn, slots):
    # levels below 10 and from 10 up go to the server's two lanes (a worker, an engine and a stream
    # each, iterating side by side); with one slot it passes from lane to lane
    srv = hn.hn_server_create(4 << 30, slots)
    try:
        reqs = []
        for j, L in enumerate([10, 6, 5, 10, 8]):
            coef, b = I.batch_problem(70 + j, L)
            reqs.append((hn.hn_mg_submit(srv, L, b, coef, prec=1), L, coef, b))
        for t, L, coef, b in reqs:
            status, x, st = hn.hn_mg_poll(srv, t, L, timeout_ns=60_000_000_000)
            assert status == hn.HN_OK
            xa, sa, _ = solve(hn, L, b, coef, prec=1)
            np.testing.assert_array_equal(x, xa)
            assert st["cycles"] == sa["cycles"]
        info = hn.hn_server_query(srv)
        assert info["completed"] == len(reqs) and info["active"] == 0 and info["queued"] == 0
        assert info["bytes_in_use"] == 0
    finally:
        hn.hn_server_destroy(srv)


@pytest.mark.parametrize("prec", [1, 2])
def test_server_reuses_device_blocks_without_leaking_state(hn, prec):
    # one slot: every request is admitted after the previous one retired, so its operator and
    # hierarchy are built in the blocks the previous request of the same level left behind
    srv = hn.hn_server_create(2 << 30, 1)
    try:
        reqs = []
        for j, L in enumerate([7, 7, 6, 7, 6, 7]):
            coef, b = I.batch_problem(40 + j, L)
            reqs.append((hn.hn_mg_submit(srv, L, b, coef if j % 3 else None, prec=prec), L,
                         coef if j % 3 else None, b))
        for t, L, coef, b in reqs:
            status, x, st = hn.hn_mg_poll(srv, t, L, timeout_ns=60_000_000_000)
            assert status == hn.HN_OK
            xa, sa, _ = solve(hn, L, b, coef, prec=prec)
            np.testing.assert_array_equal(x, xa)
            assert st["cycles"] == sa["cycles"]
        # inputs are checked when submitted
        coef, b = I.batch_problem(50, 6)
        coef = coef.copy()
        coef[3] = -1.0
        with pytest.raises(hn.HnError) as e:
            hn.hn_mg_submit(srv, 6, b, coef, prec=prec)
        assert e.value.status == hn.HN_ERR_ARG
        info = hn.hn_server_query(srv)
        assert info["completed"] == len(reqs) and info["iterations"] > 0
        assert info["iterate_ns"] > 0 and info["admit_ns"] > 0
    finally:
        hn.hn_server_destroy(srv)


def test_server_under_a_tight_budget_waits_and_releases_cached_blocks(hn):
    # a budget of 1.5 requests: the head of the queue waits for memory, and the blocks that the
    # finished request left in the cache are released to admit it; results stay those of the
    # solves alone
    L = 8
    A = hn.hn_band_create(L)
    mg = hn.hn_mg_setup(A, prec=1)
    hier = hn.hn_mg_device_bytes(mg)
    hn.hn_mg_destroy(mg)
    hn.hn_band_destroy(A)
    N = ((1 << L) + 1) ** 2
    pitch = -(-N // 128) * 128
    request = hier + 9 * pitch * 8 + (1 << L) * (1 << L) * 8 + 4096   # as the server counts it
    srv = hn.hn_server_create(int(1.5 * request), 4)
    try:
        reqs = []
        for j in range(4):
            coef, b = I.batch_problem(60 + j, L)
            reqs.append((hn.hn_mg_submit(srv, L, b, coef, prec=1), coef, b))
        for t, coef, b in reqs:
            status, x, st = hn.hn_mg_poll(srv, t, L, timeout_ns=60_000_000_000)
            assert status == hn.HN_OK
            xa, sa, _ = solve(hn, L, b, coef, prec=1)
            np.testing.assert_array_equal(x, xa)
            assert st["cycles"] == sa["cycles"]
        info = hn.hn_server_query(srv)
        assert info["completed"] == 4 and info["bytes_in_use"] == 0
    finally:
        hn.hn_server_destroy(srv)


def test_profiling_times_kernels_without_changing_results(hn):
    L = 9                  # levels 9 and 8 above the tail: separate restriction and prolongation
    b = I.rhs_uniform(L, 21)
    A = hn.hn_band_create(L)
    mg = hn.hn_mg_setup(A, prec=1)
    hn.hn_band_destroy(A)
    try:
        x0, _, _ = hn.hn_mg_solve(mg, L, b)
        tail = hn.hn_mg_get_tuning(mg)[0]
        # levels above the tail in the persistent kernels, as one launch per step, in fused sweeps
        # (the finest level's first smoothing step, its prolongation and post-smoothing apart)
        for mid, sweep, want in ((10, 0, {"mid_down", "mid_up", "tail", "outer_defect"}),
                                 (0, 0, {"jacobi", "defect", "restrict", "prolong", "tail", "outer_defect"}),
                                 (0, 1, {"jacobi_first", "jacobi", "defect", "restrict", "sweep_down",
                                         "sweep_up", "prolong", "tail", "outer_defect"}),
                                 (0, 2, {"jacobi_first", "sweep_down", "sweep_up", "prolong", "jacobi",
                                         "tail", "outer_defect"})):
            hn.hn_mg_set_tuning(mg, tail, 16, 2, 0, 1, 0, mid, sweep)
            hn.hn_mg_set_profiling(mg, True)
            x1, _, _ = hn.hn_mg_solve(mg, L, b)
            times = hn.hn_mg_kernel_times(mg)
            names = {t["name"] for t in times}
            assert want <= names, (mid, sweep, names)
            if sweep == 2:
                assert not {"defect", "restrict"} & names, names
            assert all(t["total_ms"] > 0 for t in times)
            np.testing.assert_array_equal(x0, x1)
            hn.hn_mg_set_profiling(mg, False)
    finally:
        hn.hn_mg_destroy(mg)


@pytest.mark.parametrize("mid,sweep", [(0, 0), (10, 0), (0, 1), (0, 2)])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("L", [6, 9])
def test_device_loop_skips_idle_parts_without_changing_results(hn, prec, L, mid, sweep):
    # the one-launch solve of the defect correction skips, through an IF node, the rest of a V
    # cycle after a lagged check that ends the inner solve (a check on a level run by one launch
    # per step; the persistent kernels take their checks inside and skip the rest themselves);
    # the host-driven iterations (profiling) run every kernel of every iteration.  A turn of the
    # device-side loop holds two iterations, so a solve that ends in the first may launch the
    # second's kernels as no-ops: at most one iteration's launches more than the host-driven solve.
    coef, b = I.batch_problem(5, L)
    A = hn.hn_band_create(L, coef)
    mg = hn.hn_mg_setup(A, prec=prec)
    hn.hn_band_destroy(A)
    try:
        tail = hn.hn_mg_get_tuning(mg)[0]
        hn.hn_mg_set_tuning(mg, tail, 16, 2, 0, 1, 0, mid, sweep)
        x0, st0, s0 = hn.hn_mg_solve(mg, L, b)
        n_loop = hn.hn_mg_last_launches(mg)
        hn.hn_mg_set_profiling(mg, True)
        x1, st1, s1 = hn.hn_mg_solve(mg, L, b)
        n_host = hn.hn_mg_last_launches(mg)
        hn.hn_mg_set_profiling(mg, False)
        assert s0 == s1 == hn.HN_OK
        np.testing.assert_array_equal(x0, x1)
        for k in ("cycles", "outer_iters", "inner_cycles", "relres"):
            assert st0[k] == st1[k], k
        assert 0 < n_loop <= n_host + n_host // max(1, st0["cycles"])
        if prec != 0 and L > max(tail, mid):
            assert n_loop < n_host
        # a second solve counts its own launches again
        hn.hn_mg_solve(mg, L, b)
        assert hn.hn_mg_last_launches(mg) == n_loop
    finally:
        hn.hn_mg_destroy(mg)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_launch_shapes_do_not_change_results(hn, prec):
    # the tail level, cluster size, programmatic dependent launch, bulk-copy staging, the
    # distributed shared-memory cluster levels, the prolongation fused into the first
    # post-smoothing step and the top level of the persistent kernels only change where work runs
    L = 10                 # levels 9 and 10 are large enough for the bulk-copy kernels
    coef, b = I.batch_problem(3, L)
    A = hn.hn_band_create(L, coef)
    mg = hn.hn_mg_setup(A, prec=prec)
    hn.hn_band_destroy(A)
    try:
        ref, st0, _ = hn.hn_mg_solve(mg, L, b)
        shapes = [(2, 1, 0, 0, 1, 1, 0), (4, 2, 0, 1, 1, 0, 0), (5, 16, 1, 0, 0, 1, 0), (7, 8, 2, 1, 1, 1, 0),
                  (7, 16, 2, 0, 0, 0, 0), (7, 16, 2, 0, 1, 0, 0), (6, 4, 2, 0, 1, 1, 0), (8, 16, 1, 1, 1, 0, 0),
                  (7, 16, 2, 0, 1, 1, 0), (7, 16, 2, 0, 1, 0, 10), (7, 16, 2, 0, 1, 0, 9), (7, 16, 2, 0, 1, 0, 8),
                  (5, 16, 2, 0, 1, 0, 10), (2, 1, 2, 0, 1, 0, 10), (6, 4, 0, 0, 0, 0, 10), (9, 16, 2, 0, 1, 0, 10)]
        shapes = [s + (0,) for s in shapes]
        # the fused level sweeps: every level between the tail and the finest (1; 2: and the
        # finest level's down part), with or without the prolongation fused into the finest
        # level's first post-smoothing step, without PDL
        shapes += [(7, 16, 2, 0, 1, 0, 0, 1), (2, 1, 2, 0, 1, 0, 0, 1), (5, 16, 2, 0, 1, 0, 0, 1),
                   (6, 4, 2, 0, 1, 1, 0, 1), (8, 16, 1, 0, 1, 0, 0, 1), (9, 16, 2, 0, 1, 0, 0, 1),
                   (7, 16, 0, 0, 0, 0, 0, 1), (4, 2, 3, 0, 1, 0, 0, 1),
                   (7, 16, 2, 0, 1, 0, 0, 2), (5, 16, 2, 0, 1, 0, 0, 2), (6, 4, 2, 0, 1, 1, 0, 2),
                   (9, 16, 2, 0, 1, 0, 0, 2)]
        for shape in shapes:
            hn.hn_mg_set_tuning(mg, *shape)
            assert hn.hn_mg_get_tuning(mg) == shape
            x, st, _ = hn.hn_mg_solve(mg, L, b)
            np.testing.assert_array_equal(x, ref)
            assert st["cycles"] == st0["cycles"]
        best, table = hn.hn_mg_autotune(mg, b, reps=1)
        assert best in table and len(table) == 3 * 5 * 8
        x, _, _ = hn.hn_mg_solve(mg, L, b)
        np.testing.assert_array_equal(x, ref)
    finally:
        hn.hn_mg_destroy(mg)


@pytest.mark.parametrize("coarse_L", [3, 4])
def test_other_coarse_levels_lockstep(hn, coarse_L):
    L = 7
    coef = I.lognormal_coef(L, 17)
    b = I.rhs_uniform(L, 18)
    x, st, status = solve(hn, L, b, coef, coarse_L=coarse_L, tol=0.0, max_cycles=3)
    xr, _ = O.mg_solve(L, b, coef=coef, coarse_L=coarse_L, tol=0.0, max_cycles=3)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-9
    x, st, status = solve(hn, L, b, coef, coarse_L=coarse_L, prec=1)
    assert status == hn.HN_OK and oracle_relres(L, coef, b, x) <= RELRES


def test_grouped_norm_sums_do_not_depend_on_the_schedule(hn):
    # L = 11 has 32,776 tiles: its norms are summed in two groups (two control blocks, or one
    # block group after group inside the fused tail); alone, in a batch with a small problem, and
    # with the whole cycle inside the fused tail, the results are the same bits
    L = 11
    coef, b = I.batch_problem(7, L)
    A = hn.hn_band_create(L, coef)
    mg = hn.hn_mg_setup(A, prec=1)
    hn.hn_band_destroy(A)
    c2, b2 = I.batch_problem(8, 5)
    A2 = hn.hn_band_create(5, c2)
    mg2 = hn.hn_mg_setup(A2, prec=1)
    hn.hn_band_destroy(A2)
    try:
        ref, st, status = hn.hn_mg_solve(mg, L, b)
        assert status == hn.HN_OK and oracle_relres(L, coef, b, ref) <= RELRES
        xs, stats, status = hn.hn_mg_solve_batch([mg, mg2], [L, 5], [b, b2])
        assert status == hn.HN_OK
        np.testing.assert_array_equal(xs[0], ref)
        assert stats[0]["cycles"] == st["cycles"]
        hn.hn_mg_set_tuning(mg, 11, 16, 2, 0, 1)
        x, st2, _ = hn.hn_mg_solve(mg, L, b)
        np.testing.assert_array_equal(x, ref)
        assert st2["cycles"] == st["cycles"]
    finally:
        hn.hn_mg_destroy(mg)
        hn.hn_mg_destroy(mg2)


def test_autotuned_shape_persists_through_the_cache_file(hn, tmp_path, monkeypatch):
    # HN_TUNE_CACHE: the autotuner stores its choice under (GPU, level, precision, solver, coarse
    # solver, coarse level); a later hierarchy of the same key starts with it, others do not
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("HN_TUNE_CACHE", str(path))
    L = 6
    b = I.rhs_uniform(L, 31)
    A = hn.hn_band_create(L)
    mgs = []
    try:
        mgs.append(hn.hn_mg_setup(A, prec=1))
        default = hn.hn_mg_get_tuning(mgs[0])
        mgs.append(hn.hn_mg_setup(A, prec=0))
        default64 = hn.hn_mg_get_tuning(mgs[1])
        best, table = hn.hn_mg_autotune(mgs[0], b, reps=1)
        tuned = hn.hn_mg_get_tuning(mgs[0])
        assert best == (tuned[0], tuned[1], tuned[6], tuned[7]) and len(open(path).read().splitlines()) == 1
        mgs.append(hn.hn_mg_setup(A, prec=1))
        assert hn.hn_mg_get_tuning(mgs[2]) == tuned
        mgs.append(hn.hn_mg_setup(A, prec=0))                    # another key: untouched
        assert hn.hn_mg_get_tuning(mgs[3]) == default64
        x1, _, _ = hn.hn_mg_solve(mgs[0], L, b)
        x2, _, _ = hn.hn_mg_solve(mgs[2], L, b)
        np.testing.assert_array_equal(x1, x2)
        monkeypatch.delenv("HN_TUNE_CACHE")
        mgs.append(hn.hn_mg_setup(A, prec=1))
        assert hn.hn_mg_get_tuning(mgs[4]) == default
    finally:
        for m in mgs:
            hn.hn_mg_destroy(m)
        hn.hn_band_destroy(A)
