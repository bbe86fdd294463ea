"""Pins of the learned-truncation oracle (oracle/mlp.py) against closed forms, special cases,
finite differences and brute force.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2410_09654_gb300 import inputs as I

LETTERS = "IXYZ"


def _rand_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(mlp.N_PARAMS) * scale


def test_param_layout():
    assert mlp.N_PARAMS == 128 * 80 + 128 + 128 * 128 + 128 + 128 + 1 == 27009
    p = np.arange(mlp.N_PARAMS, dtype=np.float64)
    P = mlp.unpack(p)
    assert P["W1"][1, 0] == 80 and P["b1"][0] == 128 * 80 and P["b3"][0] == mlp.N_PARAMS - 1
    assert np.array_equal(mlp.pack(P), p)


def test_features_single_z_centre():
    # Z on site 24 of 48 (0-based site 23, bin floor(16*23/48) = 7 holding sites 21..23)
    v, w = I.string("Z", 24)
    x = mlp.features([v], [w], [0.5], [0.0], 48)[0]
    assert x[0] == 1 / 48 and x[1] == 1 / 48
    assert x[2] == math.log(0.5) / 16
    for b in range(16):
        want = [2 / 3, 0, 0, 1 / 3] if b == 7 else [1, 0, 0, 0]
        assert np.allclose(x[3 + 4 * b:7 + 4 * b], want, rtol=0, atol=1e-15)
    assert not x[67:].any()


def test_features_letters_and_empty_bins():
    # N=4: sites land in bins 0, 4, 8, 12; the other twelve bins are empty (zeros)
    v, w = I.string("X", 1, "Y", 2, "Z", 4)
    x = mlp.features([v], [w], [0.0], [-2.0], 4)[0]
    assert x[0] == 3 / 4 and x[1] == 4 / 4
    assert x[2] == math.log(2.0) / 16
    want = {0: [0, 1, 0, 0], 4: [0, 0, 1, 0], 8: [1, 0, 0, 0], 12: [0, 0, 0, 1]}
    for b in range(16):
        assert list(x[3 + 4 * b:7 + 4 * b]) == want.get(b, [0, 0, 0, 0])


def test_features_random_words_by_letter_counting():
    # strings built from letter words with inputs.string (an encoding independent of the
    # oracle's bit decode); expected features counted from the words themselves
    rng = np.random.default_rng(5)
    for n in (1, 7, 16, 23, 48, 64):
        words = ["".join(rng.choice(list(LETTERS), n)) for _ in range(6)]
        words.append("I" * n)
        vs, ws, res = [], [], []
        for word in words:
            args = []
            for j, ch in enumerate(word):
                if ch != "I":
                    args += [ch, j + 1]
            v, w = I.string(*args)
            vs.append(v)
            ws.append(w)
            res.append(float(rng.uniform(0.1, 2.0)))
        x = mlp.features(vs, ws, res, [0.0] * len(vs), n)
        for r, word in enumerate(words):
            sup = [j for j, ch in enumerate(word) if ch != "I"]
            assert x[r, 0] == len(sup) / n
            assert x[r, 1] == ((sup[-1] - sup[0] + 1) / n if sup else 0.0)
            for b in range(16):
                sites = [j for j in range(n) if j * 16 // n == b]
                for t, ch in enumerate(LETTERS):
                    want = sum(word[j] == ch for j in sites) / len(sites) if sites else 0.0
                    assert abs(x[r, 3 + 4 * b + t] - want) < 1e-15


def test_forward_zero_network_is_output_bias():
    p = np.zeros(mlp.N_PARAMS)
    P = mlp.unpack(p)
    P["b3"][0] = 0.7
    z, _ = mlp.forward(p, np.random.default_rng(0).standard_normal((5, 80)))
    assert np.all(z == 0.7)


@pytest.mark.parametrize("xf", [1.5, -1.5])
def test_forward_single_path_orientation(xf):
    # one non-zero weight per layer: z = c relu(b relu(a x_f)), which fixes W1 and W2 as
    # (output, input) matrices and the ReLU placement
    p = np.zeros(mlp.N_PARAMS)
    P = mlp.unpack(p)
    f, i, j = 11, 37, 90
    P["W1"][i, f] = 2.0
    P["W2"][j, i] = -3.0
    P["w3"][j] = 0.5
    P["b2"][j] = 10.0
    X = np.zeros((1, 80))
    X[0, f] = xf
    z, _ = mlp.forward(p, X)
    want = 0.5 * max(-3.0 * max(2.0 * xf, 0.0) + 10.0, 0.0)
    assert z[0] == want


def test_forward_positive_homogeneity():
    p = _rand_params(1)
    P = mlp.unpack(p)
    P["b1"][:] = 0
    P["b2"][:] = 0
    P["b3"][:] = 0
    X = np.random.default_rng(2).standard_normal((9, 80))
    z, _ = mlp.forward(p, X)
    z3, _ = mlp.forward(p, 3.0 * X)
    assert np.allclose(z3, 3.0 * z, rtol=1e-13, atol=1e-13)
    P["w3"][:] *= -2.0
    z2, _ = mlp.forward(p, X)
    assert np.allclose(z2, -2.0 * z, rtol=1e-13, atol=1e-13)


def test_bce_closed_forms():
    assert abs(mlp.bce([0.0, 0.0], [0.0, 1.0]) - math.log(2.0)) < 1e-15
    for z in (-3.0, 0.25, 4.0):
        assert abs(mlp.bce([z], [1.0]) - math.log1p(math.exp(-z))) < 1e-15
        assert abs(mlp.bce([z], [0.0]) - math.log1p(math.exp(z))) < 1e-15
    assert abs(mlp.bce([800.0], [0.0]) - 800.0) < 1e-12  # no overflow


def test_gradient_by_finite_differences():
    rng = np.random.default_rng(3)
    p = _rand_params(4, 0.2)
    X = rng.standard_normal((6, 80))
    y = (rng.random(6) < 0.5).astype(np.float64)
    loss, g = mlp.loss_and_grad(p, X, y)
    assert abs(loss - mlp.bce(mlp.forward(p, X)[0], y)) < 1e-15
    picks = np.concatenate([rng.choice(128 * 80, 25, replace=False),
                            128 * 80 + rng.choice(128, 5, replace=False),
                            128 * 81 + rng.choice(128 * 128, 25, replace=False),
                            128 * 209 + rng.choice(128, 5, replace=False),
                            128 * 210 + rng.choice(128, 10, replace=False),
                            [mlp.N_PARAMS - 1]])
    h = 1e-6
    for k in picks:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        num = (mlp.bce(mlp.forward(pp, X)[0], y) - mlp.bce(mlp.forward(pm, X)[0], y)) / (2 * h)
        assert abs(num - g[k]) <= 1e-7 + 1e-5 * abs(num), (k, num, g[k])


def test_adam_first_steps_closed_form():
    # with a constant gradient, every bias-corrected step is -lr g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 2.0, 3.0, 4.0])
    m = np.zeros(4)
    s = np.zeros(4)
    lr = 0.01
    for t in (1, 2, 3):
        p_new, m, s = mlp.adam(p, g, m, s, t, lr)
        assert np.allclose(p_new - p, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
        p = p_new


def test_scores_zero_network_is_log_abs_after_dissipation():
    v, w = I.string("X", 1, "Y", 3)
    p = np.zeros(mlp.N_PARAMS)
    s = mlp.scores(p, [v], [w], [0.3], [-0.4], 8, gamma_dt=0.05)
    assert abs(s[0] - (math.log(0.5) - 0.05 * 2)) < 1e-15


def test_rank_values_zero_network_and_order():
    v, w = I.string("X", 1, "Y", 3)
    p = np.zeros(mlp.N_PARAMS)
    r = mlp.rank_values(p, [v], [w], [0.3], [-0.4], 8)
    assert r[0] == 0.3 * 0.3 + 0.4 * 0.4  # exactly |c|^2 when the exponent is zero
    r = mlp.rank_values(p, [v], [w], [0.3], [-0.4], 8, gamma_dt=0.05)
    assert abs(r[0] - 0.25 * math.exp(-0.2)) < 1e-16
    # a random network: rank values order the strings as the scores do (exp(2 score))
    arr = I.random_sum(4, 12, 200, kind="complex")
    q = _rand_params(6, 0.2)
    sc = mlp.scores(q, *arr, 12, gamma_dt=0.01)
    rv = mlp.rank_values(q, *arr, 12, gamma_dt=0.01)
    assert np.allclose(np.log(rv), 2 * sc, rtol=0, atol=1e-12)
    assert np.array_equal(np.argsort(-rv, kind="stable"), np.argsort(-sc, kind="stable"))


def _random_op(seed, n, m, dyadic=False):
    rng = np.random.default_rng(seed)
    keys = set()
    while len(keys) < m:
        keys.add((int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n))))
    keys = list(keys)
    v = np.array([k[0] for k in keys], np.uint64)
    w = np.array([k[1] for k in keys], np.uint64)
    if dyadic:
        re = rng.choice([0.5, -0.5, 0.25, 1.0, -1.0, 0.125], m)
        im = np.zeros(m)
    else:
        re = rng.standard_normal(m)
        im = rng.standard_normal(m)
    return v, w, re, im


@pytest.mark.parametrize("dyadic", [False, True])
def test_scored_truncation_by_log_abs_equals_abs_truncation(dyadic):
    # ranking by ln|c| keeps exactly the strings that ranking by |c| keeps, ties included
    v, w, re, im = _random_op(7, 10, 300, dyadic)
    wt = np.array([bin(int(a) | int(b)).count("1") for a, b in zip(v, w)])
    for top_k, mw, cut in ((40, -1, 0.0), (100, 12, 0.3), (7, -1, 0.0)):
        op = oracle.Op(10, v, w, re, im)
        want = oracle.truncate(op, max_weight=mw, cutoff=cut, top_k=top_k)
        got = mlp.truncate_scored(v, w, re, im, 0.5 * np.log(re * re + im * im), max_weight=mw,
                                  cutoff=cut, top_k=top_k)
        assert np.array_equal(got[0], want.v) and np.array_equal(got[1], want.w)
        assert np.array_equal(got[2], want.re) and np.array_equal(got[3], want.im)
    # with dissipation the score must include -gamma dt wt to match
    op = oracle.Op(10, v, w, re, im)
    want = oracle.truncate(op, top_k=50, gamma=0.3, dt=0.5)
    got = mlp.truncate_scored(v, w, re, im, 0.5 * np.log(re * re + im * im) - 0.15 * wt, top_k=50,
                              gamma=0.3, dt=0.5)
    assert set(zip(got[0], got[1])) == set(zip(want.v, want.w))


def test_scored_truncation_brute_force_rank_counting():
    rng = np.random.default_rng(11)
    for trial in range(20):
        m = int(rng.integers(1, 30))
        v, w, re, im = _random_op(100 + trial, 5, m, dyadic=True)
        score = rng.choice([-1.0, 0.0, 0.5, 2.0, np.nan], m)  # many exact ties
        k = int(rng.integers(1, m + 1))
        got = mlp.truncate_scored(v, w, re, im, score, top_k=k)
        kept = set(zip(got[0].tolist(), got[1].tolist()))

        def above(j, i):  # does j outrank i?
            sj, si = score[j], score[i]
            key_less = (int(v[j]), int(w[j])) < (int(v[i]), int(w[i]))
            if np.isnan(sj) and np.isnan(si):
                return key_less
            if np.isnan(sj):
                return False
            if np.isnan(si):
                return True
            return sj > si or (sj == si and key_less)

        want = {(int(v[i]), int(w[i])) for i in range(m)
                if sum(above(j, i) for j in range(m) if j != i) < k}
        assert kept == want


def test_scored_truncation_keep_set():
    v, w, re, im = _random_op(9, 8, 60)
    score = -np.arange(60, dtype=np.float64)  # index order
    keep = (v[50:53], w[50:53])
    got = mlp.truncate_scored(v, w, re, im, score, top_k=10, keep=keep)
    kept = set(zip(got[0].tolist(), got[1].tolist()))
    want = {(int(v[i]), int(w[i])) for i in list(range(10)) + [50, 51, 52]}
    assert kept == want
