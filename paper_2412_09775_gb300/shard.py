"""Data-parallel sharding of independent problems across ranks (host logic).

Every tile of a shift-variant field and every volume is an independent
reconstruction, so N GPUs split the work with no data-path collective: rank r
takes a contiguous block of tiles (row-major over the tile grid, so that a
rank's tiles are spatially adjacent and only block borders would need a halo
exchange when stitching), and timings are combined with a max over ranks.
"""
from __future__ import annotations


def tile_range(n_tiles: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of the contiguous block of tiles owned by `rank`."""
    if world < 1 or not 0 <= rank < world or n_tiles < 0:
        raise ValueError("bad rank/world/n_tiles")
    base, extra = divmod(n_tiles, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the default process group (identity for one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)
