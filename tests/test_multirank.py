"""The multi-rank host logic of bench.py on CPU: two gloo ranks on 127.0.0.1 (no GPU).

Under torchrun every rank solves its own independent problem (weak scaling, no collective on the
data path); the only collectives are the barrier around the timed region and the max of the
per-rank times.  These tests run that logic with world_size 2.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "HN_BENCH_BACKEND": "gloo"})
    import bench
    from paper_0904_4152_gb300 import inputs as I
    r, w, local, pg = bench.dist_setup(world)
    assert (r, w, local) == (rank, world, rank) and pg is not None
    bench.barrier(pg)
    t_max = bench.max_over_ranks(10.0 + rank, pg)        # per-rank timed totals (ms)
    # every rank draws its own right-hand side (independent problems)
    b = I.rhs_uniform(4, rank)
    out.put((rank, t_max, float(b.sum())))
    # the reference arm: rank 0 alone runs the oracle; the other ranks return at once
    if rank != 0:
        class A:
            steps, warmup = 1, 0
        bench.run_reference(A, rank, w, pg)
    bench.barrier(pg)
    pg.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [11.0, 11.0]            # max over ranks on both
    assert res[0][2] != res[1][2]                           # ranks solve different problems


def test_single_rank_needs_no_process_group():
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    r, w, local, pg = bench.dist_setup(1)
    assert (r, w, local, pg) == (0, 1, 0, None)
    assert bench.max_over_ranks(3.5, None) == 3.5


def test_weak_scaling_value():
    # value = all ranks' DOF / slowest rank's time
    dof, steps, world = 1_050_625, 10, 4
    t_max_ms = 25.0
    value = world * dof * steps / (t_max_ms * 1e-3)
    assert np.isclose(value, 4 * 1_050_625 * 10 / 0.025)
