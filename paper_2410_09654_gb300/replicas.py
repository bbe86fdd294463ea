"""Whole-job figures for replica runs.

The commutator path does not shard: a multi-GPU run is N independent instances, one
per GPU (one process each), with no collective on the data path.  The only
cross-rank step is the benchmark's bookkeeping: the job's time is the slowest rank's,
and the job's work is the sum of every rank's.  These helpers do that with
torch.distributed on whatever backend the process group uses (NCCL on GPUs, gloo on
CPU), and are the identity for a single process.
"""
from __future__ import annotations


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def reduce_scalar(x: float, op: str, device: str = "cuda") -> float:
    """x reduced over all ranks ("max" or "sum"); x itself without a process group."""
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
    return float(t.item())


def job_rate(units: float, ms: float, device: str = "cuda") -> tuple[float, float, float]:
    """(units of all ranks per second over the slowest rank's time, that time in ms, the
    units of all ranks) for one timed region."""
    ms_max = reduce_scalar(ms, "max", device)
    units_all = reduce_scalar(units, "sum", device)
    return units_all / (ms_max / 1e3), ms_max, units_all
