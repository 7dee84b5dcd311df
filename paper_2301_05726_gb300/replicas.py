"""Several GPUs: replicas only.

A single job does not shard: every factor links X with X xor m_k, and no
partition of the determinant keys is invariant under all excitations, so a
partitioned wavefunction would need an all-to-all exchange per factor.  What
does shard is independent work -- whole jobs of a batch, or independent theta
vectors -- with no data-path collective; ranks meet only to combine timings.
"""
from __future__ import annotations


def shard(n_items: int, rank: int, world: int) -> list:
    """Items (jobs) of this rank: round robin, every item exactly once."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return list(range(rank, n_items, world))


def combine_step(ms_local: float, units_local: float, device=None):
    """Whole-job step time and work: the slowest rank's time (max) and the
    units all ranks processed (sum).  Without an initialised process group
    the local values are returned."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms_local), float(units_local)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
