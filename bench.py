"""Benchmark: Pauli-string commutator hot path on GB300.

Timed step: one Lanczos step (A = [H, O_n] - b_n O_{n-1}, b_{n+1} = ||A||,
O_{n+1} = top-2^22(A / b_{n+1})) of the open XXZ chain on 64 sites,
H = sum X X + Y Y + 0.5 Z Z (189 strings), O_0 = sum X_i / 8, once the
operator has reached the 2^22-string cap.  `value` is [H,O] Pauli products
(|H| x |O| string products per commutator) per second; the JSON line also
carries merged strings/s, RK4 steps/s on the N=10 chain workload, the
roofline of the dominant kernel, the oracle's CPU rate and an end-to-end
figure measured through host buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 (torchrun), each rank runs an independent replica (the path does not
shard: weak scaling); value = products of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "[H,O] Pauli products/s + RK4 steps/s at ≤1e-6 rel error vs FP64 oracle"
N_SITES = 64
TOP_K = 1 << 22


def workload(top_k: int) -> str:
    cap = f"2^{top_k.bit_length() - 1}" if top_k & (top_k - 1) == 0 else str(top_k)
    return ("Lanczos on the open XXZ chain N=64 (H = sum XX+YY+0.5ZZ, 189 strings), O_0 = sum X_i/8, "
            f"top {cap} strings kept after each step; timed steps start once |O| has reached {cap}")
LATTICE_WORKLOAD = ("RK4 on the open 8x8 Heisenberg lattice (336 strings), O(0) = Z at (4,4), dt=0.02, dissipation "
                    "gamma=0.1, top 2^23 strings with trimmed stages, timed once at the cap (2 steps)")
LEARNED_WORKLOAD = ("RK4 on the open N=48 chain sum ZZ + 1.05 sum X + 0.5 sum Z (143 strings), O(0) = Z_24, "
                    "dt=0.05, 80 steps (t=4), trimmed stages; top 2^18 strings by the learned score versus by |c|, "
                    "both against the same run at top 2^22; observable Tr(O(t) Z_24)/2^N after every step")
RK4_WORKLOAD = "RK4 on the open N=10 chain sum ZZ + 1.05 sum X + 0.5 sum Z, O(0)=Z_1, dt=0.05, 40 steps, weight<=6 then |c|<1e-10"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=8)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--top-k", type=int, default=TOP_K)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-learned", action="store_true", help="skip the learned-truncation comparison")
    p.add_argument("--no-autotune", action="store_true", help="keep the default merge geometry")
    p.add_argument("--lanczos-only", action="store_true",
                   help="only the Lanczos headline (profiling runs): no RK4, lattice or pattern lines")
    p.add_argument("--merge-geometry", default=None,
                   help="BIN_TARGET,QUOTA: fix the merge geometry instead of tuning it (profiling runs)")
    p.add_argument("--lattice-only", action="store_true",
                   help="only the 8x8 lattice RK4 line (profiling runs), at --lattice-cap strings")
    p.add_argument("--lattice-cap", type=int, default=1 << 23)
    p.add_argument("--profile-window", action="store_true",
                   help="cudaProfilerStart/Stop around the first timed step (ncu --profile-from-start off)")
    return p.parse_args()


def lattice_only(args):
    """The 2D workload alone (profiling runs): ramp to the cap, one untimed step, then the timed
    steps (the first inside the profiler window when asked), then the same steps again from the
    same state with per-kernel events."""
    import torch
    from paper_2410_09654_gb300 import inputs as I, paulistr as ps
    ps.load(build_if_missing=True)
    if args.merge_geometry:
        bt, q = (int(x) for x in args.merge_geometry.split(","))
        ps.pauli_merge_geometry_fix(bt, q)
    cap = args.lattice_cap
    Hl = ps.PauliSum.from_arrays(N_SITES, *I.heisenberg_2d(8, 8).arrays())
    Ol = ps.PauliSum.from_arrays(N_SITES, *I.single(N_SITES, "Z", 28).arrays())
    pol = ps.policy(top_k=cap, gamma=0.1, trim_stages=1)
    ramp = 0
    for i in range(40):
        ps.pauli_rk4_step(Hl, Ol, 0.02, pol)
        ramp += 1
        if len(Ol) >= cap and i >= 24:
            break
    ps.pauli_rk4_step(Hl, Ol, 0.02, pol)
    start = Ol.copy()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for j in range(args.steps):
        if j == 0 and args.profile_window:
            torch.cuda.profiler.start()
        ps.pauli_rk4_step(Hl, Ol, 0.02, pol)
        if j == 0 and args.profile_window:
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    Ol = start
    ps.pauli_profile_enable(True)
    for j in range(args.steps):
        ps.pauli_rk4_step(Hl, Ol, 0.02, pol)
    prof = ps.pauli_profile_report()
    ps.pauli_profile_enable(False)
    print(json.dumps({"workload": LATTICE_WORKLOAD.replace("2^23", f"{cap}"), "profile_only": True,
                      "ramp_steps": ramp, "steps": args.steps, "ms_per_step": ms, "size": len(Ol),
                      "kernels_per_step_ms": {k: round(v[1] / args.steps, 4)
                                              for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}}), flush=True)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            # nvidia-smi takes a moment to start: wait (bounded) for its first sample, so that
            # the samples kept (those from here on) cover the timed region that follows
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None
        self.i0 = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        kept = self.lines[self.i0:] or self.lines[-1:]
        for ln in kept:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names[1:], f[5:9]):
                if val.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- workload
def workload_arrays():
    from paper_2410_09654_gb300 import inputs as I
    return I.xxz_chain(N_SITES, 0.5).arrays(), I.uniform_sum(N_SITES, "X").arrays()


def oracle_rate(top_k: int, steps: int, warmup: int, budget_s: float = 25.0):
    """The CPU oracle on a bounded sample of the same workload: the same Lanczos recursion
    with the cap lowered (2^18 strings: about a second per step on one core); returns the
    per-step (products, seconds) of the timed steps, stopping once budget_s has passed."""
    import oracle as orc
    Ha, O0a = workload_arrays()
    H = orc.Op(N_SITES, *Ha)
    prev, cur, b = orc.Op.empty(N_SITES), orc.Op(N_SITES, *O0a), 0.0
    n = 0
    while len(cur) < top_k and n < 40:  # ramp (untimed)
        b, nxt = orc.lanczos_step(H, prev, cur, b, top_k=top_k)
        prev, cur = cur, nxt
        n += 1
    rec = []
    t_all = time.perf_counter()
    for i in range(warmup + steps):
        t = time.perf_counter()
        prods = len(H) * len(cur)
        b, nxt = orc.lanczos_step(H, prev, cur, b, top_k=top_k)
        dt = time.perf_counter() - t
        prev, cur = cur, nxt
        if i >= warmup:
            rec.append((prods, dt))
        if time.perf_counter() - t_all > budget_s and len(rec) >= 1:
            break
    return rec


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sample_k = 1 << 18
    rec = oracle_rate(sample_k, args.steps, args.warmup, budget_s=150.0)
    prods = sum(p for p, _ in rec)
    secs = sum(t for _, t in rec)
    value = prods / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Pauli products/s", "n_gpus": args.gpus,
        "steps": len(rec), "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(rec), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(args.top_k), "sample": f"same recursion with the cap lowered to 2^18 strings"},
        "cpu_baseline": {"value": value, "unit": "Pauli products/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(rec)} oracle Lanczos steps at |O| = 2^18 (single-threaded C++ oracle)"},
        "e2e": {"value": value, "unit": "Pauli products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.lattice_only:
        lattice_only(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2410_09654_gb300 import inputs as I
    from paper_2410_09654_gb300 import paulistr as ps
    ps.load(build_if_missing=True)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2410_09654_gb300 import replicas as R

    def max_over_ranks(x: float) -> float:
        return R.reduce_scalar(x, "max")

    def sum_over_ranks(x: float) -> float:
        return R.reduce_scalar(x, "sum")

    Ha, O0a = workload_arrays()
    H = ps.PauliSum.from_arrays(N_SITES, *Ha)
    nH = len(Ha[0])
    pol = ps.policy(top_k=args.top_k)
    prev, cur = ps.PauliSum(N_SITES), ps.PauliSum.from_arrays(N_SITES, *O0a)
    b = 0.0
    n_done = 0
    # ramp: untimed steps until the operator has reached the cap
    while len(cur) < args.top_k and n_done < 30:
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
        n_done += 1
    ramp_steps = n_done
    # merge geometry for this size class, picked by timing the candidates (untimed)
    if args.merge_geometry:
        bt, q = (int(x) for x in args.merge_geometry.split(","))
        ps.pauli_merge_geometry_fix(bt, q)
        tune = {"bin_target": bt, "quota": q, "fixed": True}
    else:
        tune = None if args.no_autotune else ps.pauli_autotune_commutator(H, cur, reps=2)
    for _ in range(args.warmup):
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
        n_done += 1

    # host snapshots of the first end-to-end states: the recursion steps ahead from here while
    # each input state is downloaded, then restarts from device copies of the first one, so
    # that the timed loop and the end-to-end leg run the same states (the recursion is
    # deterministic)
    snaps = []
    start = (prev.copy(), cur.copy(), b)  # the timed and the profiled region both start here
    start_step = n_done + 1               # index n of the first timed b_n
    if not args.no_e2e:
        for _ in range(max(1, min(args.steps, 4))):
            snaps.append((prev.download(), cur.download(), b))
            b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
    # untimed pass over the same K steps: the library's block cache then holds every buffer
    # size these steps use, as in a long run whose sizes have settled
    prev, cur, b = start[0].copy(), start[1].copy(), start[2]
    for _ in range(args.steps):
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
    prev, cur, b = start[0].copy(), start[1].copy(), start[2]

    # ---------------------------------------------------------------- timed region
    # K Lanczos steps, un-instrumented; the per-kernel CUDA-event timings come from a second
    # pass over the same K steps, restarted from the same device state (events recorded by the
    # library on each kernel's launching stream), so that event recording does not slow the
    # headline and the per-kernel times describe exactly the timed steps.
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    products = 0
    merged = 0
    contributions = 0
    groups = split_groups = 0
    bs = []
    barrier()
    clocks.start()
    launches0 = ps.pauli_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        products += nH * len(cur)
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
        st = ps.pauli_last_merge_stats()
        merged += st["merged"]
        contributions += st["contributions"]
        groups += st["groups"]
        split_groups += st["split_groups"]
        bs.append(b)
    ev1.record(stream)
    barrier()
    launches = ps.pauli_launch_count() - launches0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    value, ms_max, products_all = R.job_rate(products, ms)
    merged_rate = sum_over_ranks(merged) / (ms_max / 1e3)
    contrib_rate = sum_over_ranks(contributions) / (ms_max / 1e3)

    # per-kernel durations over the same K steps again, from the same start state (events on)
    prev, cur, b = start[0].copy(), start[1].copy(), start[2]
    prof_bs = []
    ps.pauli_profile_enable(True)
    barrier()
    prof_products = 0
    prof_contrib = 0
    prof_merged = 0
    evp0 = torch.cuda.Event(enable_timing=True)
    evp1 = torch.cuda.Event(enable_timing=True)
    evp0.record(stream)
    prof_src = 0
    for _ in range(args.steps):
        prof_products += nH * len(cur)
        prof_src += len(prev)  # O_{n-1} enters the merge as a source term
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
        prof_bs.append(b)
        st = ps.pauli_last_merge_stats()
        prof_contrib += st["contributions"]
        prof_merged += st["merged"]
    evp1.record(stream)
    barrier()
    prof = ps.pauli_profile_report()
    ps.pauli_profile_enable(False)
    prof_ms = evp0.elapsed_time(evp1)
    assert prof_bs == bs, "the profiled pass must repeat the timed steps"
    del start

    # ---------------------------------------------------------------- roofline of the dominant kernel
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    top = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("none", (1, 1.0))
    kname, (klaunch, kms) = top
    avg_s = kms / 1e3 / max(klaunch, 1)
    roof = {"kernel": kname, "share": kms / max(sum(v[1] for v in prof.values()), 1e-9)}
    per_step = {k: (v[0] / args.steps, v[1] / args.steps) for k, v in prof.items()}
    entries = (prof_contrib + prof_src) / args.steps  # merge entries per launch
    if kname.startswith("k_merge"):
        if kname.endswith("_f"):
            # full contribution records: each entry (32 B) read once, each merged string written once
            alg = entries * 32 + (prof_merged / args.steps) * 32
        else:
            # 8-byte references read once, each referenced operand record (32 B) gathered once
            alg = entries * (8 + 32) + (prof_merged / args.steps) * 32
        roof.update({"bound": "hbm", "achieved": alg / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "peak_kind": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), kernel timed inside the step",
                     "algorithmic_bytes_per_launch": alg, "entries_per_launch": entries})
        tr = dram_traffic(kname)
        if tr is not None:
            roof["traffic"] = tr["bytes_per_unit"] * entries
            roof["traffic_source"] = tr["source"]
    elif kname == "k_emit_products":
        # each operand string (32 B record + 4 B hash) read once, each contribution record
        # (32 B) written once; the pair tests are table lookups, not the bound
        alg = (prof_products / args.steps / nH) * 36 + (prof_contrib / args.steps) * 32
        alg /= max(klaunch / args.steps, 1)
        roof.update({"bound": "hbm", "achieved": alg / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "peak_kind": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), kernel timed inside the step",
                     "algorithmic_bytes_per_launch": alg})
        tr = dram_traffic(kname)
        if tr is not None:
            roof["traffic"] = tr["bytes_per_unit"] * prof_contrib / max(klaunch, 1)
            roof["traffic_source"] = tr["source"]
    else:
        roof.update({"bound": "hbm", "achieved": None, "peak": hbm_peak, "unit": "GB/s"})
    if roof.get("achieved") is not None:
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof.setdefault("traffic", None)

    # ---------------------------------------------------------------- end to end (host buffers)
    e2e = None
    if snaps:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        host = [([pin(x) for x in sp], [pin(x) for x in sc], sb) for sp, sc, sb in snaps]
        e_prev, e_cur = ps.PauliSum(N_SITES, args.top_k), ps.PauliSum(N_SITES, args.top_k)
        # pinned host buffers receiving each step's new operator O_{n+1} (storage order)
        out_host = [torch.empty(args.top_k, dtype=dt).pin_memory()
                    for dt in (torch.int64, torch.int64, torch.float64, torch.float64)]
        barrier()
        t0 = time.perf_counter()
        e_prod = 0
        h2d = d2h = 0
        for hp, hc, sb in host:  # the timed loop's first states, each from host arrays
            e_prev.upload(*hp)
            e_cur.upload(*hc)
            # the product operand into the merge's hash order (canonical order is slower); O_{n-1}
            # enters the merge as a source term, whose emission does not depend on its order
            e_cur.sort_by_hash()
            e_prod += nH * len(hc[0])
            h2d += 32 * (len(hc[0]) + len(hp[0]))
            ps.pauli_lanczos_step(H, e_prev, e_cur, sb, pol)  # b_n read back to the host
            # O_{n+1} back to pinned host memory, written there by the library's unpacking kernel
            res = ps.pauli_sum_download_device(e_cur, out=out_host)
            d2h += 8 + 32 * int(res[2].numel())
            torch.cuda.current_stream().synchronize()
        barrier()
        t_e2e = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": sum_over_ranks(e_prod) / t_e2e, "unit": "Pauli products/s",
               "h2d_bytes_per_step": int(h2d / len(host)), "d2h_bytes_per_step": int(d2h / len(host)),
               "states": f"the first {len(host)} input states of the timed loop, uploaded from pinned host arrays",
               "api": "pauli_sum_upload x2 (pinned host arrays, read by the packing kernel over the host link) + "
                      "pauli_sum_sort_by_hash of O_n + pauli_lanczos_step (b_n to host) + pauli_sum_download_device of "
                      "O_{n+1} into pinned host arrays"}

    if args.lanczos_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "Pauli products/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                              "profile_only": True, "kernels_per_step_ms": {k: round(v[1], 4) for k, v in per_step.items()},
                              "merge_groups_per_step": groups / args.steps,
                              "merge_split_groups_per_step": split_groups / args.steps,
                              "launches_before_timed": launches0, "gpu_launches": launches,
                              "roofline": roof, "e2e": e2e}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    # ---------------------------------------------------------------- RK4 steps/s (N=10 chain)
    n10 = 10
    Hr = ps.PauliSum.from_arrays(n10, *I.tilted_ising_chain(n10).arrays())
    Z1 = I.single(n10, "Z", 1).arrays()
    rk_pol = ps.policy(max_weight=6, cutoff=1e-10)
    Or = ps.PauliSum.from_arrays(n10, *Z1)
    for _ in range(40):  # untimed warm-up: the same trajectory once (the operator grows every step)
        ps.pauli_rk4_step(Hr, Or, 0.05, rk_pol)
    Or = ps.PauliSum.from_arrays(n10, *Z1)
    Z1s = ps.PauliSum.from_arrays(n10, *Z1)
    barrier()
    t0 = time.perf_counter()
    obs = []
    for _ in range(40):
        ps.pauli_rk4_step(Hr, Or, 0.05, rk_pol)
        obs.append(ps.pauli_trace_product(Or, Z1s).real)
    barrier()
    t_rk = max_over_ranks(time.perf_counter() - t0)
    rk4 = {"steps_per_s": sum_over_ranks(40) / t_rk, "workload": RK4_WORKLOAD, "final_size": len(Or),
           "observable_t2": obs[-1]}

    # ---------------------------------------------------------------- RK4 on the 8x8 lattice
    # the 2D workload (336-string H, beyond 256 order codes) at its cap
    lat_cap = 1 << 23
    Hl = ps.PauliSum.from_arrays(N_SITES, *I.heisenberg_2d(8, 8).arrays())
    Ol = ps.PauliSum.from_arrays(N_SITES, *I.single(N_SITES, "Z", 28).arrays())
    lat_pol = ps.policy(top_k=lat_cap, gamma=0.1, trim_stages=1)
    for i in range(40):  # ramp (untimed) until the cap holds
        ps.pauli_rk4_step(Hl, Ol, 0.02, lat_pol)
        if len(Ol) >= lat_cap and i >= 24:
            break
    # merge geometry for the lattice's size class (untimed), unless fixed or disabled
    lat_tune = None
    if not args.merge_geometry and not args.no_autotune:
        lat_tune = ps.pauli_autotune_commutator(Hl, Ol, reps=1)
    lat_prod = 0
    barrier()
    evl0 = torch.cuda.Event(enable_timing=True)
    evl1 = torch.cuda.Event(enable_timing=True)
    evl0.record(stream)
    for _ in range(2):
        lat_prod += 4 * len(Hl) * len(Ol)  # four commutators per step
        ps.pauli_rk4_step(Hl, Ol, 0.02, lat_pol)
    evl1.record(stream)
    barrier()
    t_lat = max_over_ranks(evl0.elapsed_time(evl1)) / 1e3
    rk4_lattice = {"workload": LATTICE_WORKLOAD, "ms_per_step": 1e3 * t_lat / 2,
                   "steps_per_s": sum_over_ranks(2) / t_lat, "products_per_s": sum_over_ranks(lat_prod) / t_lat,
                   "size": len(Ol), "merge_geometry_autotuned": lat_tune}

    # ---------------------------------------------------------------- FP32 coefficients (2D lattice)
    f32_res = None
    if not args.no_learned:
        f32_res = lattice_f32(stream, Hl, Ol, lat_pol)

    # ---------------------------------------------------------------- batched disorder realisations
    batch_res = None
    if not args.no_learned:
        batch_res = batched_instances(stream, fixed_geometry=bool(args.merge_geometry))
        batch_res["full_caps"] = batched_instances_full(stream)

    # ---------------------------------------------------------------- learned truncation
    learned_res = None
    if not args.no_learned:
        learned_res = learned_truncation(stream, peaks_bf16=float(peaks.get("bf16_tflops", 1900.0)))

    # ---------------------------------------------------------------- CPU oracle baseline
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rec = oracle_rate(1 << 18, 16, 1, budget_s=15.0)
        cp = sum(p for p, _ in rec) / sum(t for _, t in rec)
        cpu = {"value": cp, "unit": "Pauli products/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(rec)} Lanczos steps of the same recursion with the cap lowered to 2^18 strings "
                         f"(single-threaded C++ oracle)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Pauli products/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(args.top_k), "n_sites": N_SITES, "H_strings": nH, "top_k": args.top_k,
                       "ramp_steps": ramp_steps, "merge_geometry_autotuned": tune,
                       "l2": f"inputs larger than L2: |O| = {args.top_k} strings x 32 B = {args.top_k * 32 / 1e6:.0f} MB per operand; the merge "
                       f"bins hold {contributions / args.steps * 32 / 1e9:.1f} GB of contribution records per step "
                       "(L2 is 129 MB)", "parallelism": "replicas" if world > 1 else "single"},
            "merged_strings_per_s": merged_rate,
            "contributions_per_s": contrib_rate,
            "contributions_per_step": contributions / args.steps,
            "merge_groups_per_step": groups / args.steps, "merge_split_groups_per_step": split_groups / args.steps,
            "timed_steps_n": [start_step, start_step + args.steps - 1],
            "b_n_timed": bs,
            "rk4": rk4,
            "rk4_lattice": rk4_lattice,
            "rk4_lattice_f32": f32_res,
            "batched_instances": batch_res,
            "learned_truncation": learned_res,
            "roofline": roof,
            "kernels_per_step_ms": {k: round(v[1], 4) for k, v in sorted(per_step.items(), key=lambda kv: -kv[1][1])},
            "profiled_region_ms_per_step": prof_ms / args.steps,
            "profiled_region": "the timed steps again, from the same device state, with per-kernel CUDA events",
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "launches_before_timed": launches0,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


BATCH_WORKLOAD = ("RK4 of 512 disorder realisations of the random-field XXZ chain N=32 (125 strings: XX+YY+ZZ bonds "
                  "+ h_i Z_i, h_i ~ U[-W, W] from SplitMix64 seeded 20241012 + instance, W = 0.5 / 2 / 5 for instances "
                  "0-170 / 171-341 / 342-511), O(0) = Z_16, dt=0.05, trimmed stages, uneven per-instance caps "
                  "2^(8 + instance mod 7) (256 to 16384; the description's 2^14-2^20 scaled down 64x), timed once "
                  "every instance has run 12 steps")


def batched_instances(stream, n_inst: int = 512, ramp: int = 12, timed: int = 3, loop_sample: int = 32,
                      fixed_geometry: bool = False):
    """All instances in one tagged sum (pauli_batch_rk4_step) against the single-instance
    path looped over a sample of the instances (scaled to all): instance-steps/s and
    products/s of both.  Under N ranks each rank takes the instances b with b mod N = rank
    (independent problems, no exchange); rates are the ranks' sums over the slowest rank."""
    import torch
    from paper_2410_09654_gb300 import inputs as I, paulistr as ps, replicas as R
    n, shift = 32, 32
    N = shift + 9
    mine = R.instance_share(n_inst)       # this rank's instances (global ids)
    W = [0.5 if b <= 170 else (2.0 if b <= 341 else 5.0) for b in range(n_inst)]
    Hs = [I.random_field_xxz_chain(n, W[b], b).arrays() for b in mine]
    caps = np.array([1 << (8 + b % 7) for b in mine], np.int64)
    m = len(mine)
    hcoef = np.stack([h[2] for h in Hs])
    Hc = ps.PauliSum.from_arrays(N, Hs[0][0], Hs[0][1], np.ones(len(Hs[0][0])), np.zeros(len(Hs[0][0])))
    B = ps.PauliBatch(Hc, hcoef, shift, caps)
    z = I.single(n, "Z", 16).arrays()
    v = np.array([int(z[0][0]) | (j << shift) for j in range(m)], np.uint64)
    O = ps.PauliSum.from_arrays(N, v, np.zeros(m, np.uint64), np.ones(m), np.zeros(m))
    for _ in range(ramp):
        ps.pauli_batch_rk4_step(B, Hc, O, 0.05, trim_stages=1)
    tune = None if fixed_geometry else ps.pauli_autotune_commutator(Hc, O, reps=2)  # batched commutators
    sizes = ps.pauli_batch_counts(B, O)
    prod = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(timed):
        prod += 4 * len(Hs[0][0]) * len(O)
        ps.pauli_batch_rk4_step(B, Hc, O, 0.05, trim_stages=1)
    torch.cuda.synchronize()
    t_b = R.reduce_scalar((time.perf_counter() - t0) / timed, "max")
    prod = R.reduce_scalar(prod, "sum")
    # the single-instance path on a sample spread over the caps and disorder strengths
    pick = np.linspace(0, m - 1, min(loop_sample, m)).astype(int)
    t_loop, prod_loop = 0.0, 0
    for b in pick:
        H = ps.PauliSum.from_arrays(n, *Hs[b])
        Ob = ps.PauliSum.from_arrays(n, *z)
        pol = ps.policy(top_k=int(caps[b]), trim_stages=1)
        for _ in range(ramp):
            ps.pauli_rk4_step(H, Ob, 0.05, pol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(timed):
            prod_loop += 4 * len(Hs[b][0]) * len(Ob)
            ps.pauli_rk4_step(H, Ob, 0.05, pol)
        torch.cuda.synchronize()
        t_loop += time.perf_counter() - t0
    scale = m / len(pick)
    t_loop_all = R.reduce_scalar(t_loop / timed * scale, "max")  # seconds per step of this rank's instances, looped
    prod_loop = R.reduce_scalar(prod_loop, "sum")
    t_loop = R.reduce_scalar(t_loop, "max")
    return {"workload": BATCH_WORKLOAD, "instances": n_inst, "strings": int(R.reduce_scalar(sizes.sum(), "sum")),
            "strings_per_instance_min_max": [int(R.reduce_scalar(sizes.min(), "min")), int(R.reduce_scalar(sizes.max(), "max"))],
            "batched": {"ms_per_step": 1e3 * t_b, "instance_steps_per_s": n_inst / t_b,
                        "products_per_s": prod / timed / t_b},
            "looped_single_instance": {"ms_per_step": 1e3 * t_loop_all, "instance_steps_per_s": n_inst / t_loop_all,
                                       "products_per_s": prod_loop / t_loop * 1.0,
                                       "sample": f"{loop_sample} instances spread over the caps, scaled to {n_inst}"},
            "speedup": t_loop_all / t_b, "merge_geometry_autotuned": tune,
            "ranks": R.world(), "instances_per_rank": "b mod ranks = rank",
            "not_built": "one persistent graph-captured launch: each step is a sequence of launches with host "
                         "synchronisation on data-dependent sizes"}


BATCH_FULL_WORKLOAD = ("the same 512 realisations with the description's caps 2^(14 + instance mod 7) (16384 to "
                       "1048576 strings), in groups of instances whose caps add up to at most 2^22 (one tagged sum "
                       "and one pauli_batch per group, so that a merge's entry bound stays within its budget); "
                       "timed once every instance has run 16 steps")


def batched_instances_full(stream, n_inst: int = 512, ramp: int = 16, timed: int = 2, group_cap: int = 1 << 22):
    """The batched realisations at the full per-instance caps, grouped by cap, against the
    single-instance path looped over two instances of every cap (scaled to all).  Under N
    ranks each rank takes the instances b with b mod N = rank."""
    import torch
    from paper_2410_09654_gb300 import inputs as I, paulistr as ps, replicas as R
    n, shift = 32, 32
    W = [0.5 if b <= 170 else (2.0 if b <= 341 else 5.0) for b in range(n_inst)]
    caps = np.array([1 << (14 + b % 7) for b in range(n_inst)], np.int64)
    z = I.single(n, "Z", 16).arrays()
    mine = R.instance_share(n_inst)
    # groups: instances sorted by cap, filled greedily up to group_cap strings of caps
    order = sorted(mine, key=lambda b: (caps[b], b))
    groups, cur, tot = [], [], 0
    for b in order:
        if cur and tot + caps[b] > group_cap:
            groups.append(cur)
            cur, tot = [], 0
        cur.append(b)
        tot += caps[b]
    if cur:
        groups.append(cur)
    runs = []
    for g in groups:
        tb = max(1, (len(g) - 1).bit_length())
        N = shift + tb
        Hs = [I.random_field_xxz_chain(n, W[b], b).arrays() for b in g]
        Hc = ps.PauliSum.from_arrays(N, Hs[0][0], Hs[0][1], np.ones(len(Hs[0][0])), np.zeros(len(Hs[0][0])))
        B = ps.PauliBatch(Hc, np.stack([h[2] for h in Hs]), shift, caps[g])
        v = np.array([int(z[0][0]) | (j << shift) for j in range(len(g))], np.uint64)
        O = ps.PauliSum.from_arrays(N, v, np.zeros(len(g), np.uint64), np.ones(len(g)), np.zeros(len(g)))
        runs.append((B, Hc, O, len(Hs[0][0])))
    for _ in range(ramp):
        for B, Hc, O, _nh in runs:
            ps.pauli_batch_rk4_step(B, Hc, O, 0.05, trim_stages=1)
    strings = sum(len(O) for _, _, O, _ in runs)
    prod = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(timed):
        for B, Hc, O, nh in runs:
            prod += 4 * nh * len(O)
            ps.pauli_batch_rk4_step(B, Hc, O, 0.05, trim_stages=1)
    torch.cuda.synchronize()
    t_b = R.reduce_scalar((time.perf_counter() - t0) / timed, "max")
    prod = R.reduce_scalar(prod, "sum")
    strings = R.reduce_scalar(strings, "sum")
    n_groups = R.reduce_scalar(len(groups), "sum")
    del runs
    # single-instance path: two instances of every cap class, scaled by the class sizes
    t_loop_all, prod_loop, t_loop = 0.0, 0, 0.0
    per_class = {}
    for c in range(7):
        members = [b for b in mine if b % 7 == c]
        if not members:
            continue
        t_c = 0.0
        for b in (members[0], members[len(members) // 2]):
            H = ps.PauliSum.from_arrays(n, *I.random_field_xxz_chain(n, W[b], b).arrays())
            Ob = ps.PauliSum.from_arrays(n, *z)
            pol = ps.policy(top_k=int(caps[b]), trim_stages=1)
            for _ in range(ramp):
                ps.pauli_rk4_step(H, Ob, 0.05, pol)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(timed):
                prod_loop += 4 * len(H) * len(Ob)
                ps.pauli_rk4_step(H, Ob, 0.05, pol)
            torch.cuda.synchronize()
            dt_ = time.perf_counter() - t0
            t_c += dt_
            t_loop += dt_
        t_loop_all += t_c / 2 / timed * len(members)
        per_class[str(1 << (14 + c))] = 1e3 * t_c / 2 / timed * len(members)
    t_loop_all = R.reduce_scalar(t_loop_all, "max")
    prod_loop = R.reduce_scalar(prod_loop, "sum")
    t_loop = R.reduce_scalar(t_loop, "max")
    return {"workload": BATCH_FULL_WORKLOAD, "instances": n_inst, "groups": int(n_groups), "strings": int(strings),
            "batched": {"ms_per_step": 1e3 * t_b, "instance_steps_per_s": n_inst / t_b,
                        "products_per_s": prod / timed / t_b},
            "looped_single_instance": {"ms_per_step": 1e3 * t_loop_all, "instance_steps_per_s": n_inst / t_loop_all,
                                       "products_per_s": prod_loop / t_loop,
                                       "sample": "two instances per cap class, scaled to the 512",
                                       "ms_per_step_by_cap": per_class},
            "speedup": t_loop_all / t_b}


F32_WORKLOAD = ("RK4 on the open 8x8 Heisenberg lattice (336 strings), O(0) = Z at (4,4), dt=0.02, dissipation "
                "gamma=0.1, top 2^20 strings with trimmed stages, 30 steps (t=0.6) from O(0), with FP64 coefficients, "
                "FP32 coefficients (FP64 accumulation of exact products) and FP32 arithmetic with compensated sums "
                "(H and O rounded to FP32; FP64 norms); step times also at the 2^23 cap from the FP64 run's state")


def lattice_f32(stream, Hl, Ol, lat_pol, steps: int = 30):
    """The 2D workload run with FP64, FP32 and compensated-FP32 coefficients from the same start:
    the error of each FP32 mode per observable (autocorrelation Tr(O(t) Z_c)/2^N and ||O(t)||),
    the step times of the study, and the step times at the 2^23 cap (two steps from the FP64
    lattice run's state at the cap, converted to each precision)."""
    import torch
    from paper_2410_09654_gb300 import inputs as I, paulistr as ps
    pol = ps.policy(top_k=1 << 20, gamma=0.1, trim_stages=1)
    Ha = I.heisenberg_2d(8, 8).arrays()
    Oa = I.single(N_SITES, "Z", 28).arrays()
    pv, pw = I.string("Z", 28)
    probe = (np.array([pv], np.uint64), np.array([pw], np.uint64))
    at_cap = {}
    for name, prec in (("f64", ps.PS_COEF_F64), ("f32", ps.PS_COEF_F32), ("f32c", ps.PS_COEF_F32C)):
        Hp = Hl.copy().set_precision(prec)
        Op_ = Ol.copy().set_precision(prec)
        ps.pauli_rk4_step(Hp, Op_, 0.02, lat_pol)  # untimed: the cache holds this precision's sizes
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            ps.pauli_rk4_step(Hp, Op_, 0.02, lat_pol)
        e1.record(stream)
        e1.synchronize()
        at_cap[name] = e0.elapsed_time(e1) / 2
        del Hp, Op_
    runs = {}
    for name, prec in (("f64", ps.PS_COEF_F64), ("f32", ps.PS_COEF_F32), ("f32c", ps.PS_COEF_F32C)):
        H = ps.PauliSum.from_arrays(N_SITES, *Ha).set_precision(prec)
        O = ps.PauliSum.from_arrays(N_SITES, *Oa).set_precision(prec)
        obs, nrm = [], []
        t_steps = 0.0
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ps.pauli_rk4_step(H, O, 0.02, pol)
            e1.record(stream)
            e1.synchronize()
            t_steps += e0.elapsed_time(e1)
            obs.append(ps.pauli_coefficients(O, *probe)[0].real)
            nrm.append(ps.pauli_norm(O))
        runs[name] = (np.array(obs), np.array(nrm), t_steps / steps, len(O))
    a64, n64, t64, s64 = runs["f64"]
    out = {"workload": F32_WORKLOAD, "ms_per_step_at_2p23_cap": at_cap,
           "ms_per_step": {k: v[2] for k, v in runs.items()}, "final_size": {k: v[3] for k, v in runs.items()},
           "autocorrelation_final": {k: float(v[0][-1]) for k, v in runs.items()}}
    for name in ("f32", "f32c"):
        a, nrm = runs[name][0], runs[name][1]
        out[name + "_error_vs_f64"] = {
            "autocorrelation_abs_max": float(np.max(np.abs(a - a64))),
            "autocorrelation_rel_max": float(np.max(np.abs(a - a64) / np.abs(a64))),
            "norm_rel_max": float(np.max(np.abs(nrm - n64) / n64))}
    out["note"] = ("f32: FP32 values, exact products accumulated in FP64; f32c: FP32 products and "
                   "Sum2-compensated FP32 sums; both store FP32 values in the 32-byte records")
    return out


def learned_truncation(stream, peaks_bf16: float, lg_cap: int = 18, steps: int = 80, iters: int = 4000):
    """Train the BF16 scorer on the method's own runs (cap M versus 4M, labels 10 steps ahead)
    and compare the observable error of learned and plain truncation at cap M against a run at
    16M; also the scoring kernel's time and tensor throughput inside the learned run."""
    import torch
    from paper_2410_09654_gb300 import inputs as I, learned as L, paulistr as ps
    n = 48
    M = 1 << lg_cap
    H = ps.PauliSum.from_arrays(n, *I.tilted_ising_chain(n).arrays())
    O0 = ps.PauliSum.from_arrays(n, *I.single(n, "Z", 24).arrays())
    pv, pw = I.string("Z", 24)
    probe = (np.array([pv], np.uint64), np.array([pw], np.uint64))
    dt = 0.05
    pol = ps.policy(top_k=M, trim_stages=1)
    ref, t_ref = L.rk4_observable(H, O0, dt, steps, ps.policy(top_k=16 * M, trim_stages=1), probe)
    plain, t_plain = L.rk4_observable(H, O0, dt, steps, pol, probe)
    t0 = time.perf_counter()
    data = L.collect(H, O0, dt, M, [10, 20, 30, 40, 50, 60], 10)
    t1 = time.perf_counter()
    model = ps.PauliMLP(n, seed=1)
    loss0 = L.mean_loss(model, data)
    batch = 16384
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    L.train(model, data, iters, batch=batch, lr=1e-3)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    loss1 = L.mean_loss(model, data)
    mlp, t_mlp = L.rk4_observable(H, O0, dt, steps, pol, probe, model=model)
    ps.pauli_profile_enable(True)  # a second pass with per-kernel events (its wall time is not used)
    L.rk4_observable(H, O0, dt, steps, pol, probe, model=model)
    prof = ps.pauli_profile_report()
    ps.pauli_profile_enable(False)
    e_pl = np.abs(plain[:, 0] - ref[:, 0])
    e_ml = np.abs(mlp[:, 0] - ref[:, 0])
    # plain truncation at larger caps: the cap it needs to reach the learned error at M
    larger = {}
    for f in (2, 4):
        obs_f, t_f = L.rk4_observable(H, O0, dt, steps, ps.policy(top_k=f * M, trim_stages=1), probe)
        larger[f * M] = (float(np.abs(obs_f[:, 0] - ref[:, 0]).mean()), 1e3 * t_f)
    equal = None
    for cap_f, (err_f, ms_f) in sorted(larger.items()):
        if err_f <= float(e_ml.mean()):
            equal = {"plain_cap": cap_f, "plain_ms_per_step": ms_f, "learned_ms_per_step": 1e3 * t_mlp,
                     "speedup_at_equal_error": ms_f / (1e3 * t_mlp)}
            break
    fwd_launches, fwd_ms = prof.get("k_mlp_fwd", (0, 0.0))
    cand = [len(C) for C, _ in data]
    # the scoring kernel alone on the last candidate set (strings per launch known exactly)
    C_last = data[-1][0]
    ps.pauli_mlp_scores(model, C_last, 0.0)
    ps.pauli_profile_enable(True)
    for _ in range(5):
        ps.pauli_mlp_scores(model, C_last, 0.0)
    kprof = ps.pauli_profile_report()
    ps.pauli_profile_enable(False)
    flop_per_string = 2 * (80 * 128 + 128 * 128 + 128)
    kl, kms = kprof.get("k_mlp_fwd", (0, 0.0))
    fwd_roof = None
    if kl:
        achieved = len(C_last) * flop_per_string / (kms / 1e3 / kl) / 1e12
        fwd_roof = {"kernel": "k_mlp_fwd_tc", "bound": "tensor", "achieved": achieved, "peak": peaks_bf16,
                    "unit": "TFLOP/s", "frac": achieved / peaks_bf16,
                    "peak_kind": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json bf16_tflops), kernel timed alone",
                    "flop_per_string": flop_per_string, "strings_per_launch": len(C_last),
                    "ms_per_launch": kms / kl}
    return {
        "workload": LEARNED_WORKLOAD, "cap": M, "reference_cap": 16 * M,
        "observable_error_mean": {"plain": float(e_pl.mean()), "learned": float(e_ml.mean())},
        "observable_error_max": {"plain": float(e_pl.max()), "learned": float(e_ml.max())},
        "ms_per_step": {"plain": 1e3 * t_plain, "learned": 1e3 * t_mlp, "reference": 1e3 * t_ref},
        "plain_at_larger_caps": {str(k): {"observable_error_mean": e, "ms_per_step": t} for k, (e, t) in larger.items()},
        "equal_error": equal,
        "training": {"candidates": int(sum(cand)), "positive_fraction": L.positive_fraction(data),
                     "label": "kept in the top 2^18 of the 2^20 run 10 steps later",
                     "iterations": iters, "batch": batch, "lr": 1e-3, "loss_before": loss0, "loss_after": loss1,
                     "seconds": t3 - t2, "samples_per_s": iters * batch / (t3 - t2), "collect_seconds": t1 - t0},
        "scorer_ms_per_step": fwd_ms / steps,
        "scorer_roofline": fwd_roof,
        "kernel": "scorer: tcgen05.mma kind::f16 (bf16 operands in shared memory, fp32 accumulators in tensor memory); "
                  "training: mma.sync m16n8k16 bf16",
    }


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")
KERNEL_SOURCE = os.path.join(ROOT, "paper_2410_09654_gb300", "csrc", "merge.cu")


def dram_traffic(kname: str):
    """DRAM bytes per unit of work measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum
    of the captured launch over its units: merge entries for the merge, contribution records
    for the emission), from the committed capture summary; None when the kernel source has
    changed since the capture (sha1 of merge.cu recorded beside it)."""
    import hashlib
    if not os.path.exists(TRAFFIC_FILE):
        return None
    sha = hashlib.sha1(open(KERNEL_SOURCE, "rb").read()).hexdigest()
    for line in open(TRAFFIC_FILE):
        if line.startswith("#"):
            continue
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("kernel") == kname and f.get("merge_cu_sha1") == sha:
            return {"bytes_per_unit": float(f["dram_bytes_per_unit"]), "source": f.get("capture", "")}
    return None

if __name__ == "__main__":
    main()
