"""Window sharding of the matvec over ranks (one process per GPU).

The extended ANOVA kernel is the mean of L independent per-window Gauss
transforms (Sec. 3, Eq. discrete_ANOVA), so a rank that holds a contiguous
range of the windows computes its share of Gamma_full x and one sum over the
ranks completes it.  Every rank holds the full N-vectors; the Krylov scalars
are then computed redundantly from identical vectors.

window_range assigns the ranges; allreduce_sum is the reduce callback a
window-range plan calls (nlh_reduce_fn) to sum its share in place, on the
stream of the library call, with torch.distributed (NCCL on GPUs, gloo on
CPU tensors).
"""
from __future__ import annotations


def window_range(L: int, world: int, rank: int):
    """(first, count) of the windows of `rank`: contiguous ranges, sizes
    differing by at most one, the larger ones first; every window belongs
    to exactly one rank.  Ranks beyond L get an empty range (count 0 is not
    a valid plan range, so callers need world <= L)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d of world %d" % (rank, world))
    base, extra = divmod(L, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def allreduce_sum(buf, stream=None) -> None:
    """Sum `buf` in place over all ranks of the default process group, issued
    on `stream` (a torch stream; None = the current one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return
    if stream is None or not buf.is_cuda:
        dist.all_reduce(buf)
        return
    with torch.cuda.stream(stream):
        dist.all_reduce(buf)
