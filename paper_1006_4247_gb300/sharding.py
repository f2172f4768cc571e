"""Host logic of runs on several GPUs (one process per GPU).

Disorder samples are independent Markov chains (each has its own couplings),
so the path shards by sample with no exchange of data between ranks: every
rank simulates its own samples, drawn from coupling seeds no other rank uses,
with its own Philox seed.  Ranks meet only to time the run: a barrier on both
sides of the timed region and the maximum of the elapsed times.  The reported
throughput is the work of all ranks divided by that maximum (weak scaling:
the per-rank work is fixed as ranks are added).
"""
from __future__ import annotations

SEED_STRIDE = 100000  # coupling-seed offset between ranks (> samples per rank)
ENGINE_SEED0 = 7


def coupling_seed0(base: int, rank: int) -> int:
    """First coupling seed of `rank`'s samples; ranks use disjoint ranges as
    long as a rank has fewer than SEED_STRIDE samples."""
    return base + SEED_STRIDE * rank


def engine_seed(rank: int) -> int:
    """Philox seed of `rank`'s engine."""
    return ENGINE_SEED0 + rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over the ranks of the default process group (the
    value itself when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device_sync=None) -> None:
    """Barrier over the ranks (if a group exists), then the optional device
    synchronisation."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
    if device_sync is not None:
        device_sync()


def weak_throughput(units_per_step_per_rank: float, steps: int, world: int, elapsed: float, scale: float) -> float:
    """Units of all ranks per unit time: units_per_step * steps * world /
    (elapsed * scale), elapsed the maximum over ranks."""
    if elapsed <= 0:
        raise ValueError("elapsed time must be positive")
    return units_per_step_per_rank * steps * world / (elapsed * scale)
