"""Sharding of history ranges over ranks (one process per GPU).

Histories are independent (the paper's Sec. 4 notes that MC is task parallel),
and every history's random numbers are keyed by its global id, so ranks only
need disjoint id ranges; the per-rank integer tallies then add up exactly to
the single-GPU tally.  The optional combine step is one sum-reduction after
the run (never inside the transport).
"""
from __future__ import annotations


def history_range(rank: int, world: int, step: int, n_per_rank: int) -> tuple[int, int]:
    """[first, first + n) of global history ids for `rank` in benchmark step
    `step`: step-major, rank-minor, so that ranks and steps never overlap."""
    if not (0 <= rank < world) or n_per_rank < 0 or step < 0:
        raise ValueError("bad rank/world/step")
    first = (step * world + rank) * n_per_rank
    return first, n_per_rank


def split(n_total: int, world: int) -> list[tuple[int, int]]:
    """Contiguous split of [0, n_total) into `world` ranges (sizes differ by at most 1)."""
    out, start = [], 0
    for r in range(world):
        n = n_total // world + (1 if r < n_total % world else 0)
        out.append((start, n))
        start += n
    return out


def combine_tallies(tensors, op_sum=True):
    """Sum per-rank tallies in place across the default process group
    (int64 integer tallies add exactly; float64 second moments add too)."""
    import torch.distributed as dist

    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return tensors
