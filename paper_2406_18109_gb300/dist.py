"""Multi-rank helpers for weak scaling (one process per GPU).

Independent work units (Black-Scholes batches) are sharded by giving every
rank its own batch: there is no collective on the data path.  The only
cross-rank communication is control: the slowest rank's time and the total
number of units, combined after the timed region.
"""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank r's batch: the configured seed on rank 0, distinct elsewhere."""
    return base_seed if rank == 0 else base_seed + 1000 * rank


def combine(ms_local: float, units_local: float, device=None):
    """(value, ms_max, units_total): whole-job throughput in units/s over all
    ranks, timed by the slowest rank.  Works with gloo (CPU) or NCCL."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return units_local / (ms_local / 1e3), ms_local, units_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    units = float(u.item())
    return units / (ms / 1e3), ms, units
