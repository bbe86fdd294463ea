"""Replica runs on more than one GPU: the path does not shard, so N ranks run independent
instances and only the benchmark's bookkeeping crosses ranks (max time, summed work).
Checked here with two gloo ranks on CPU, and the reference arm's rank handling under a
two-rank environment."""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2410_09654_gb300 import replicas as R
        # rank r did (r + 1) * 1000 units in (r + 1) * 10 ms
        value, ms_max, units = R.job_rate((rank + 1) * 1000.0, (rank + 1) * 10.0, device="cpu")
        out[rank] = (value, ms_max, units, R.reduce_scalar(rank + 0.5, "max", device="cpu"))
    finally:
        dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, ms_max, units, mx = res[rank]
        assert ms_max == 20.0                 # the slowest rank's time
        assert units == 3000.0                # work of both ranks
        assert value == pytest.approx(3000.0 / 0.020)
        assert mx == 1.5


def test_job_rate_single_process_is_identity():
    from paper_2410_09654_gb300 import replicas as R
    assert R.job_rate(500.0, 4.0, device="cpu") == (500.0 / 0.004, 4.0, 500.0)


def test_reference_arm_runs_on_rank0_only():
    # under a two-rank launch the non-zero rank exits at once without output
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_json_contract():
    # rank 0 prints exactly one JSON line with the contract's keys (the oracle on the host)
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_instance_share_partitions_the_instances():
    # the batched realisations are split over ranks without an exchange: every instance on
    # exactly one rank, shares of equal size up to one, and every cap class (b mod 7) on each
    from paper_2410_09654_gb300 import replicas as R
    n = 512
    for w in (1, 2, 3, 4, 8):
        shares = [R.instance_share(n, r, w) for r in range(w)]
        flat = sorted(b for sh in shares for b in sh)
        assert flat == list(range(n))
        sizes = [len(sh) for sh in shares]
        assert max(sizes) - min(sizes) <= 1
        for sh in shares:
            assert {b % 7 for b in sh} == set(range(7))
    assert R.instance_share(n) == list(range(n))  # one process: every instance
