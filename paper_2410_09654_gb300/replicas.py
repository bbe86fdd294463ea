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


def world() -> int:
    dist = _dist()
    return 1 if dist is None else dist.get_world_size()


def rank() -> int:
    dist = _dist()
    return 0 if dist is None else dist.get_rank()


def instance_share(n_inst: int, r: int | None = None, w: int | None = None) -> list[int]:
    """The independent instances (disorder realisations) rank r runs out of n_inst: every
    instance b with b mod w == r, so that the caps, which cycle with b, spread evenly."""
    r = rank() if r is None else r
    w = world() if w is None else w
    return [b for b in range(n_inst) if b % w == r]


def reduce_scalar(x: float, op: str, device: str = "cuda") -> float:
    """x reduced over all ranks ("max", "min" or "sum"); x itself without a process group."""
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "min": dist.ReduceOp.MIN, "sum": dist.ReduceOp.SUM}[op])
    return float(t.item())


def job_rate(units: float, ms: float, device: str = "cuda") -> tuple[float, float, float]:
    """(units of all ranks per second over the slowest rank's time, that time in ms, the
    units of all ranks) for one timed region."""
    ms_max = reduce_scalar(ms, "max", device)
    units_all = reduce_scalar(units, "sum", device)
    return units_all / (ms_max / 1e3), ms_max, units_all
