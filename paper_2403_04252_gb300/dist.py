"""Multi-GPU host logic of the propagation: one process per GPU, impact parameters sharded across ranks.

Every straight-line path is independent (the paper runs one MPI rank per impact parameter), so the data
path has no collective at all: each rank propagates its own paths with the library.  The only
collectives are host-side: the maximum of the per-rank timings (a benchmark reports the slowest rank)
and the gather of per-path observables to rank 0, which forms the cross sections with the library's
wpccc_cross_sections (paper_2403_04252_gb300.cross_sections).  They go through
torch.distributed, so the same code runs on NCCL (one GPU per rank) and on gloo (CPU tests).
"""
from __future__ import annotations

import numpy as np

__all__ = ["shard_impact_parameters", "max_over_ranks", "gather_paths"]


def shard_impact_parameters(b0: float, b1: float, per_rank: int, rank: int, world: int) -> np.ndarray:
    """This rank's impact parameters of a scan of per_rank * world values uniform in [b0, b1]:
    every world-th value starting at `rank`, so that each rank gets the same number of paths (weak
    scaling: the work per GPU is fixed) spread over the whole range, and the union is the full scan."""
    if world < 1 or not 0 <= rank < world or per_rank < 1:
        raise ValueError("need world >= 1, 0 <= rank < world, per_rank >= 1")
    return np.linspace(b0, b1, per_rank * world)[rank::world].copy()


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over all ranks (x itself without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_paths(b: np.ndarray, values: np.ndarray, device=None):
    """Gather every rank's (impact parameters, per-path values) to rank 0, sorted by impact parameter.
    Returns (b_all, values_all) on rank 0 and (None, None) elsewhere; ranks may hold different counts."""
    import torch
    import torch.distributed as dist
    b = np.asarray(b, dtype=np.float64)
    values = np.asarray(values, dtype=np.float64).reshape(b.size, -1)
    if not (dist.is_available() and dist.is_initialized()):
        order = np.argsort(b, kind="stable")
        return b[order], values[order]
    world, rank = dist.get_world_size(), dist.get_rank()
    n = torch.tensor([b.size], dtype=torch.int64, device=device)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n)
    counts = [int(c.item()) for c in counts]
    width = 1 + values.shape[1]
    nmax = max(counts)
    mine = np.zeros((nmax, width))
    mine[:b.size, 0] = b
    mine[:b.size, 1:] = values
    buf = torch.as_tensor(mine, device=device)
    bufs = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf)
    if rank != 0:
        return None, None
    rows = np.concatenate([bufs[k].cpu().numpy()[:counts[k]] for k in range(world)])
    order = np.argsort(rows[:, 0], kind="stable")
    return rows[order, 0], rows[order, 1:]
