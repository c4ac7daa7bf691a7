"""Row-sharded sketching across ranks, on CPU: two gloo ranks on 127.0.0.1.

Each rank sketches its contiguous block of rows with their global indices and
one sum all-reduce combines the partials (paper_2409_14309_gb300.sharded).  The
per-rank sketch is injected (the oracle's CountSketch of the rank's rows at
their global indices, the role snsolve_sketch_rows plays on a GPU), so what is
tested here is the partition, the global indexing and the collective: on
integer-valued data every partial sum is exact in FP64, so the combined sketch
must equal the single-process oracle sketch bit for bit."""
import os
import socket
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M, N, D, SEED = 1001, 7, 64, 9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data():
    rng = np.random.default_rng(77)
    return (rng.integers(-50, 51, size=(M, N)).astype(np.float64),
            rng.integers(-50, 51, size=M).astype(np.float64))


def _oracle_rows(A_local, b_local, row0, d, kind, seed):
    """The oracle's CountSketch of rows row0.. at their global indices."""
    from oracle import hashing as H
    rows = A_local.shape[0]
    h, s = H.countsketch_hash(seed, row0 + rows, d)
    h, s = h[row0:], s[row0:]
    SA = np.zeros((d, A_local.shape[1]))
    Sb = np.zeros(d)
    np.add.at(SA, h, s[:, None] * A_local.numpy())
    np.add.at(Sb, h, s * b_local.numpy())
    return torch.from_numpy(SA), torch.from_numpy(Sb)


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2409_14309_gb300 import sharded
    A, b = _data()
    row0, rows = sharded.row_partition(M, world, rank)
    aug = sharded.sharded_sketch(None, torch.from_numpy(A[row0:row0 + rows]), torch.from_numpy(b[row0:row0 + rows]),
                                 row0, D, seed=SEED, local_sketch=_oracle_rows)
    dist.destroy_process_group()
    q.put((rank, row0, rows, aug.numpy()))


def test_two_ranks_sum_to_the_whole_sketch():
    sys.path.insert(0, ROOT)
    from oracle import sketch as OS
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=120) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    A, b = _data()
    ref = np.column_stack([OS.countsketch_apply(A, D, SEED), OS.countsketch_apply(b, D, SEED)])
    assert [(g[1], g[2]) for g in got] == [(0, 501), (501, 500)]
    for _, _, _, aug in got:
        assert np.array_equal(aug, ref)


def test_row_partition_covers_rows_once():
    sys.path.insert(0, ROOT)
    from paper_2409_14309_gb300 import sharded
    for m, world in [(10, 3), (1 << 20, 8), (7, 7), (5, 8)]:
        parts = [sharded.row_partition(m, world, r) for r in range(world)]
        assert parts[0][0] == 0
        for (r0, c0), (r1, _) in zip(parts, parts[1:]):
            assert r0 + c0 == r1
        assert sum(c for _, c in parts) == m
        assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
