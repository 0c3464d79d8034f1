"""Rank helpers for running the solver on several GPUs (one process per GPU).

Slices are independent problems once the readout is decoupled (Sec. II.A), so ranks
never exchange data on the solve path: each rank reconstructs its own slices, and the
only collectives are timing reductions.  Works with the nccl and gloo backends.
"""
from __future__ import annotations


def slice_shard(nslices: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [start, start + count) of the slices rank `rank` reconstructs when a
    scan's `nslices` slices are split over `world` ranks.  The first nslices % world
    ranks take one slice more, so no rank waits on a last, partly filled wave of
    another (the load-balance lesson of Sec. VI.B)."""
    if world < 1 or not (0 <= rank < world) or nslices < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(nslices, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def _reduce(value: float, op_name: str) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(value: float) -> float:
    """Largest value over all ranks (wall times: the job ends with its slowest rank)."""
    return _reduce(value, "MAX")


def sum_over_ranks(value: float) -> float:
    """Sum over all ranks (work units)."""
    return _reduce(value, "SUM")
