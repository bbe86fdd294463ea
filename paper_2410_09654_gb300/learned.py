"""Learned truncation workflow on top of the library's calls: gather training data from the
method's own runs, train the scorer, and measure what it changes in an observable.

Orchestration only: every arithmetic step (RK4 steps, candidate capture, labels, the
network's forward and backward passes, Adam, truncation, observables) is a library call.

Training data (one reading of "trained on the method's runs at cap M versus a larger
cap"): a run at cap M exposes, at chosen steps s, its candidate set C_s (the step's result
before the final top-M trim).  A run at cap 4M gives, at step s + horizon, its top-M
strings T.  A candidate's label is whether it belongs to T: whether the more accurate run
still ranks the string among its M most important ones a few steps later.
"""
from __future__ import annotations

import time

import numpy as np

from . import paulistr as ps


def rk4_observable(H, O0, dt: float, n_steps: int, pol, probe, model=None, stream=None):
    """Run n_steps RK4 steps from a copy of O0 and return the probe strings' coefficients
    after every step (complex array [n_steps, n_probe]) and the mean wall time per step."""
    O = O0.copy()
    pv, pw = probe
    out = np.empty((n_steps, len(pv)), np.complex128)
    t_total = 0.0
    for k in range(n_steps):
        t0 = time.perf_counter()
        if model is None:
            ps.pauli_rk4_step(H, O, dt, pol)
        else:
            ps.pauli_rk4_step_mlp(H, O, dt, pol, model=model)
        out[k] = ps.pauli_coefficients(O, pv, pw)  # synchronises
        t_total += time.perf_counter() - t0
    return out, t_total / max(n_steps, 1)


def collect(H, O0, dt: float, top_k: int, sample_steps, horizon: int, big_factor: int = 4, trim_stages: int = 1):
    """[(candidates C_s, labels y_s)] for s in sample_steps (see the module docstring)."""
    import torch
    n = O0.n_sites
    last = max(sample_steps)
    pol_s = ps.policy(top_k=top_k, trim_stages=trim_stages)
    pol_b = ps.policy(top_k=big_factor * top_k, trim_stages=trim_stages)
    pol_t = ps.policy(top_k=top_k)
    A = O0.copy()
    cands = {}
    for step in range(1, last + 1):
        C = ps.PauliSum(n) if step in sample_steps else None
        ps.pauli_rk4_step_mlp(H, A, dt, pol_s, cand_out=C)
        if C is not None:
            cands[step] = C
    B = O0.copy()
    data = []
    for step in range(1, last + horizon + 1):
        ps.pauli_rk4_step(H, B, dt, pol_b)
        s = step - horizon
        if s in cands:
            T = B.copy()
            ps.pauli_truncate(T, pol_t)
            data.append((cands[s], ps.pauli_mlp_labels(cands[s], T)))
    torch.cuda.synchronize()
    return data


def train(model, data, n_iter: int, batch: int = 16384, lr: float = 1e-3, seed: int = 0, log_every: int = 0):
    """Adam on random contiguous batches of the candidate sets; returns the logged losses."""
    rng = np.random.default_rng(seed)
    sizes = np.array([len(C) for C, _ in data], np.int64)
    weights = sizes / sizes.sum()
    losses = []
    for it in range(n_iter):
        j = int(rng.choice(len(data), p=weights))
        C, y = data[j]
        nb = int(min(batch, sizes[j]))
        i0 = int(rng.integers(0, sizes[j] - nb + 1))
        want = bool(log_every) and (it % log_every == 0 or it == n_iter - 1)
        loss = ps.pauli_mlp_train_step(model, C, y, i0, nb, lr, want_loss=want)
        if want:
            losses.append((it, loss))
    return losses


def mean_loss(model, data) -> float:
    """Mean BCE of the model over all candidates of data."""
    tot, cnt = 0.0, 0
    for C, y in data:
        _, l = ps.pauli_mlp_gradient(model, C, y, 0, len(C))
        tot += l * len(C)
        cnt += len(C)
    return tot / max(cnt, 1)


def positive_fraction(data) -> float:
    s = sum(float(y.sum().item()) for _, y in data)
    return s / max(sum(len(C) for C, _ in data), 1)


def scorer_workload(cap_log2: int = 18, steps: int = 40, reps: int = 3, seed: int = 1) -> int:
    """The scorer's and the trainer's kernels on real candidates: RK4 on the N=48 chain
    sum ZZ + 1.05 sum X + 0.5 sum Z from Z_24 (dt 0.05, trimmed stages, cap 2^cap_log2) for
    `steps` steps keeping the last step's candidates, then `reps` scorings of all of them
    and `reps` training steps on the first 16384.  Returns the number of candidates."""
    import torch
    from . import inputs as I
    n = 48
    H = ps.PauliSum.from_arrays(n, *I.tilted_ising_chain(n).arrays())
    O = ps.PauliSum.from_arrays(n, *I.single(n, "Z", 24).arrays())
    pol = ps.policy(top_k=1 << cap_log2, trim_stages=1)
    C = ps.PauliSum(n)
    for _ in range(steps):
        ps.pauli_rk4_step_mlp(H, O, 0.05, pol, cand_out=C)
    model = ps.PauliMLP(n, seed=seed)
    g = torch.Generator(device="cuda").manual_seed(seed)
    y = (torch.rand(len(C), device="cuda", generator=g) < 0.5).float()
    for _ in range(reps):
        ps.pauli_mlp_scores(model, C, 0.0)
    for _ in range(reps):
        ps.pauli_mlp_train_step(model, C, y, 0, min(16384, len(C)), 1e-3)
    torch.cuda.synchronize()
    return len(C)
