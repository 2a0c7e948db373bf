"""Replica timing across ranks: the path does not shard (each rank advances
its own mesh, no data exchange), so a multi-GPU run is N independent
replicas; the only collectives are the barrier around the timed region and
the maximum of the ranks' times."""


def job_time_ms(ms_local, device=None):
    """Largest of the ranks' times (ms); the local time when not distributed.
    Uses the process group's backend (NCCL with CUDA tensors, gloo on CPU)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms_local)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, ms_job, world):
    """Units processed by all ranks per second (weak scaling: every rank
    processes the same work)."""
    return world * units_per_rank * steps / (ms_job / 1e3)
