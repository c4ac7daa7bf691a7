"""Row-sharded sketch-and-solve over several processes (one GPU each).

The sketch is linear in the rows of [A | b], and every row keeps its global
index in the counter-based hash stream, so S [A | b] is the sum over ranks of
each rank's sketch of its own rows (snsolve_sketch_rows).  One all-reduce of
the d x (n+1) partials (torch.distributed, NCCL on GPUs) gives every rank the
full sketch; the small FP64 QR and back-solve then run replicated
(snsolve_solve_sketched), so every rank holds x^.

Only marshalling and the collective live here: the sketch and the solve are
the library's kernels.  `local_sketch` can replace the per-rank sketch (it
must return the rank's partial (SA, Sb) for its global rows), which is how the
collective logic is tested on CPU ranks.
"""
import torch
import torch.distributed as dist


def row_partition(m, world, rank):
    """(row0, rows) of `rank` when m rows are split into `world` contiguous
    blocks whose sizes differ by at most one."""
    base, extra = divmod(int(m), int(world))
    row0 = rank * base + min(rank, extra)
    return row0, base + (1 if rank < extra else 0)


def sharded_sketch(ctx, A_local, b_local, row0, d, kind="countsketch", seed=0, group=None, local_sketch=None):
    """[SA | Sb] of the whole row-sharded matrix on every rank (d x (n+1)):
    this rank's partial sketch of rows row0.., then one sum all-reduce."""
    if local_sketch is None:
        SA, Sb = ctx.sketch_rows(A_local, b_local, row0, d, kind=kind, seed=seed)
    else:
        SA, Sb = local_sketch(A_local, b_local, row0, d, kind, seed)
    aug = torch.cat([SA, Sb.reshape(-1, 1)], dim=1).contiguous()
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(aug, op=dist.ReduceOp.SUM, group=group)
    return aug


def sharded_lstsq(ctx, A_local, b_local, row0, d, kind="countsketch", seed=0, group=None):
    """Sketch-and-solve of a row-sharded problem: x^ on every rank."""
    aug = sharded_sketch(ctx, A_local, b_local, row0, d, kind=kind, seed=seed, group=group)
    return ctx.solve_sketched(aug)
