"""Data-parallel sharding of a point batch across ranks (one GPU per rank).

Points are independent (each rank solves its own slice, no data-path
collective); the initial guess of a point depends only on its global index
(hj_solver_opts.point_offset), so a sharded run reproduces the unsharded one.
The only cross-rank traffic is the timing/count reduction of the benchmark.
"""
import torch
import torch.distributed as dist


def weak_offset(rank, per_rank):
    """Global index of the first point of `rank` when every rank solves `per_rank` points."""
    return rank * per_rank


def strong_slice(rank, world, B):
    """[lo, hi) of a B-point batch split as evenly as possible over `world` ranks."""
    q, r = divmod(B, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def reduce_step_stats(times_ms, counts, device=None):
    """Max over ranks of each time and sum over ranks of each count (the
    benchmark's whole-job aggregation).  Works on any initialised backend;
    without a process group it returns the inputs."""
    t = torch.tensor([float(v) for v in times_ms], dtype=torch.float64, device=device)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()], [float(v) for v in c.tolist()]
