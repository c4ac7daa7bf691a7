"""The N > 1 bench path on CPU: replicas (one problem per rank, different data
per rank), timing = the slowest rank, value = all ranks' solves / that time.
Two gloo ranks on 127.0.0.1."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]                       # the second rank is slower
    worst = bench.max_over_ranks(ms, "cpu", world)
    rate = bench.whole_job_rate(10, world, worst)
    dist.destroy_process_group()
    q.put((rank, worst, rate))


def test_two_ranks_take_the_slowest_and_count_all_solves():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, worst, rate in got:
        assert worst == 20.0
        assert rate == pytest.approx(10 * 2 / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, "cpu", 1) == 7.0
    assert bench.whole_job_rate(4, 1, 8.0) == pytest.approx(500.0)


def test_ranks_solve_different_problems():
    """Each rank's replica gets its own data (weak scaling, no shared rows)."""
    sys.path.insert(0, ROOT)
    import bench
    from synth import ill_conditioned_problem
    a0, _, _ = ill_conditioned_problem(64, 4, seed=bench.DATA_SEED, kappa=10.0, noise=1e-3)
    a1, _, _ = ill_conditioned_problem(64, 4, seed=bench.DATA_SEED + 1000, kappa=10.0, noise=1e-3)
    assert not np.array_equal(a0, a1)
