"""CPU oracle of the learned truncation scorer and of truncation by an arbitrary score.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it; the CUDA
library never does, and the two share no code.

The paper's conclusion proposes predicting the importance of Pauli strings with
machine learning instead of ranking them by |c| alone; it does not fix a model.
This library's definition, followed here in plain numpy FP64 (no BF16 rounding):

* Features of a string s = (v, w) with coefficient c on N sites (80 inputs):
  x[0] = wt(s)/N with wt = popcount(v|w) (the Pauli weight of the dissipation
  section); x[1] = extent/N, extent = last - first + 1 over the non-identity sites
  (0 for the identity); x[2] = ln(max(|c|, 1e-300))/16; x[3 + 4b + t] = the fraction
  of the sites of bin b (site j, 0-based, lies in bin floor(16 j / N)) whose letter
  is t, t = 0..3 for I, X, Y, Z (Z bit v, X bit w: I=(0,0), X=(0,1), Y=(1,1),
  Z=(1,0)); an empty bin gives zeros; x[67..79] = 0.
* Network: z = w3 . relu(W2 relu(W1 x + b1) + b2) + b3, W1 128x80, W2 128x128
  (rows = outputs).
* Loss: binary cross-entropy on the logit z, averaged over the batch.
* Update: Adam (Kingma and Ba), bias-corrected.
* Score used to rank strings for truncation: ln|c| - gamma dt wt + z, i.e. ln|c|
  after the dissipation factor e^{-gamma dt wt}, shifted by the learned logit;
  with z = 0 it orders strings exactly as |c| does.

Flat parameter layout (FP32 on the device, FP64 here): W1 (128*80, row-major),
b1 (128), W2 (128*128, row-major), b2 (128), w3 (128), b3 (1).

Parity: every function here is pinned by ``tests/test_mlp_oracle.py`` (features by
per-site letter counting, the network by closed-form special cases and positive
homogeneity, gradients by central finite differences of the forward pass, Adam by
its closed-form first step, the scored truncation by brute force and by its
reduction to the pinned |c| truncation of ``oracle.truncate``; rank values by their
closed form for a zero network and their order against the scores).
"""
from __future__ import annotations

import math

import numpy as np

N_FEAT = 80
N_USED = 67
HID = 128
N_BINS = 16
SHAPES = [("W1", (HID, N_FEAT)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("w3", (HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 27009
LOG_FLOOR = 1e-300


def unpack(p: np.ndarray) -> dict:
    """Views of the flat parameter vector, by name."""
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def features(v: np.ndarray, w: np.ndarray, re: np.ndarray, im: np.ndarray, n_sites: int) -> np.ndarray:
    """The 80 inputs of each string (definition in the module docstring)."""
    v = np.asarray(v, np.uint64)
    w = np.asarray(w, np.uint64)
    m = len(v)
    x = np.zeros((m, N_FEAT), np.float64)
    bins = [(16 * j) // n_sites for j in range(n_sites)]
    per_bin = np.bincount(bins, minlength=N_BINS).astype(np.float64)
    for r in range(m):
        vv, ww = int(v[r]), int(w[r])
        sup = [j for j in range(n_sites) if ((vv | ww) >> j) & 1]
        x[r, 0] = len(sup) / n_sites
        x[r, 1] = (sup[-1] - sup[0] + 1) / n_sites if sup else 0.0
        a = math.hypot(float(re[r]), float(im[r]))
        x[r, 2] = math.log(max(a, LOG_FLOOR)) / 16.0
        counts = np.zeros((N_BINS, 4))
        for j in range(n_sites):
            t = ((vv >> j) & 1) * 2 + ((ww >> j) & 1)  # (z, x): 0 I, 1 X, 3 Y, 2 Z
            letter = {0: 0, 1: 1, 3: 2, 2: 3}[t]
            counts[bins[j], letter] += 1
        for b in range(N_BINS):
            if per_bin[b] > 0:
                x[r, 3 + 4 * b:3 + 4 * b + 4] = counts[b] / per_bin[b]
    return x


def forward(p: np.ndarray, X: np.ndarray):
    """Logits z (one per row of X) and the activations the backward pass needs."""
    P = unpack(p)
    a1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ P["w3"] + P["b3"][0]
    return z, (X, a1, h1, a2, h2)


def bce(z: np.ndarray, y: np.ndarray) -> float:
    """Mean binary cross-entropy of logits z against labels y in {0, 1}."""
    z = np.asarray(z, np.float64)
    y = np.asarray(y, np.float64)
    per = np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))
    return float(per.mean()) if len(per) else 0.0


def loss_and_grad(p: np.ndarray, X: np.ndarray, y: np.ndarray):
    """(mean BCE, gradient of it with respect to the flat parameters) by backpropagation."""
    P = unpack(p)
    z, (X, a1, h1, a2, h2) = forward(p, X)
    n = len(z)
    dz = (1.0 / (1.0 + np.exp(-z)) - np.asarray(y, np.float64)) / n
    g = {"w3": h2.T @ dz, "b3": np.array([dz.sum()])}
    dh2 = np.outer(dz, P["w3"]) * (a2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ P["W2"]) * (a1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    return bce(z, y), pack(g)


def adam(p, g, m, s, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One bias-corrected Adam update (step number t >= 1); returns new (p, m, s)."""
    m = beta1 * m + (1.0 - beta1) * g
    s = beta2 * s + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    sh = s / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(sh) + eps), m, s


def scores(p: np.ndarray, v, w, re, im, n_sites: int, gamma_dt: float = 0.0) -> np.ndarray:
    """ln|c| - gamma dt wt + z for every string (the ranking quantity of learned truncation)."""
    X = features(v, w, re, im, n_sites)
    z, _ = forward(p, X)
    wt = np.array([bin(int(a) | int(b)).count("1") for a, b in zip(v, w)], np.float64)
    a2 = np.asarray(re, np.float64) ** 2 + np.asarray(im, np.float64) ** 2
    with np.errstate(divide="ignore"):
        return 0.5 * np.log(a2) - gamma_dt * wt + z  # -inf for c = 0


def rank_values(p: np.ndarray, v, w, re, im, n_sites: int, gamma_dt: float = 0.0) -> np.ndarray:
    """|c|^2 e^{2 (z - gamma dt wt)} = exp(2 score): the same order as ``scores`` without a
    logarithm, and exactly |c|^2 when the exponent is zero (the ranking quantity the library
    computes for learned truncation)."""
    X = features(v, w, re, im, n_sites)
    z, _ = forward(p, X)
    wt = np.array([bin(int(a) | int(b)).count("1") for a, b in zip(v, w)], np.float64)
    q = np.asarray(re, np.float64) ** 2 + np.asarray(im, np.float64) ** 2
    e = 2.0 * (z - gamma_dt * wt)
    return np.where(e == 0.0, q, q * np.exp(e))


def truncate_scored(v, w, re, im, score, max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0,
                    gamma: float = 0.0, dt: float = 0.0, keep=None):
    """Truncation with the top-k ranked by a given score instead of |c| (dissipation, weight
    filter, exact-zero drop and strict cutoff as in ``oracle.truncate``); exact score ties keep
    the smaller key (v, then w, unsigned); keep-set strings are never dropped; a NaN score
    ranks below every number.  Returns (v, w, re, im) sorted by key."""
    v = np.asarray(v, np.uint64)
    w = np.asarray(w, np.uint64)
    re = np.array(re, np.float64)
    im = np.array(im, np.float64)
    score = np.asarray(score, np.float64)
    wt = np.array([bin(int(a) | int(b)).count("1") for a, b in zip(v, w)], np.int64)
    if gamma != 0.0:
        f = np.array([math.exp(-((gamma * dt) * float(k))) for k in range(65)])
        re = re * f[wt]
        im = im * f[wt]
    ok = ~((re == 0.0) & (im == 0.0))
    if max_weight >= 0:
        ok &= wt <= max_weight
    if cutoff > 0.0:
        ok &= ~(re * re + im * im < cutoff * cutoff)
    idx = np.nonzero(ok)[0]
    if top_k > 0 and len(idx) > top_k:
        nan = np.isnan(score[idx])
        s = np.where(nan, -np.inf, score[idx])
        # sort: score descending (NaN last), then v, w ascending
        order = sorted(range(len(idx)), key=lambda j: (nan[j], -s[j], int(v[idx[j]]), int(w[idx[j]])))
        top = set(idx[j] for j in order[:top_k])
        kset = set()
        if keep is not None:
            kset = set(zip((int(a) for a in keep[0]), (int(b) for b in keep[1])))
        idx = np.array([i for i in idx if i in top or (int(v[i]), int(w[i])) in kset], np.int64)
    o = sorted(idx.tolist(), key=lambda i: (int(v[i]), int(w[i])))
    o = np.array(o, np.int64)
    return v[o], w[o], re[o], im[o]
