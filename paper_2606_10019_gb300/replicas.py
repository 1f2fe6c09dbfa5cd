"""Host logic of a run on several GPUs: every rank registers its own
independent problems (no data exchange), and the job's throughput is the
units all ranks processed divided by the slowest rank's time."""
from __future__ import annotations


def rank_stream(base_stream: int, rank: int) -> int:
    """Seed stream of a rank's scenes and trajectory: independent problems
    per rank."""
    return base_stream + 100 * rank


def combine(units: float, seconds: float, device=None) -> tuple[float, float]:
    """(units summed over ranks, seconds maximised over ranks); the identity
    when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()), float(t.item())
