"""One sky on several GPUs: the particle paste partitioned by particle index.

Every rank holds the whole halo catalogue (the solve is per halo and cheap) and a contiguous
share of the particles; it assigns and deposits its share into its own full-size map planes
(y, b and their compensation planes), and one all-reduce (sum) of the planes gives every rank
the map of all particles.  The halo paste is partitioned the same way, by halo index.  The
deposit is linear in the particles, so the sum of the ranks' maps is the map of the whole sky
up to the rounding of the final sum (hi and lo planes are summed separately; hi + lo is the
value).  Host logic only: the kernels are those of one GPU.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of the items of rank `rank` among `world` ranks: contiguous, sizes differing
    by at most one, in rank order, covering [0, n) exactly once."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError(f"shard_range: n={n}, rank={rank}, world={world}")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def map_planes(n_planes: int, n_maps: int, ny: int, nx: int, device):
    """One contiguous FP32 buffer [n_planes, n_maps, ny, nx] (zeroed): the planes of several
    map pairs, reduced across ranks in one collective."""
    import torch

    return torch.zeros((n_planes, n_maps, ny, nx), dtype=torch.float32, device=device)


def reduce_maps(buf, world: int):
    """Sum the ranks' map planes in place (one all-reduce over the whole buffer)."""
    if world <= 1:
        return buf
    import torch.distributed as dist

    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    return buf
