"""Pins of the multi-word oracle (oracle/multiword.py, masks of any width): equality with the
single-word C++ oracle for N <= 64, dense matrices on local supports that straddle the word
boundary at site 64, and invariance under moving an operator by whole words.  CPU only."""
import math

import numpy as np
import pytest

import oracle as orc
from oracle import dense
from oracle import multiword as mw
from paper_2410_09654_gb300 import inputs as I


def _terms(arrays):
    v, w, re, im = arrays
    return [((int(a), int(b)), complex(c, d)) for a, b, c, d in zip(v, w, re, im)]


def _as_dict(op):
    return {(int(a), int(b)): complex(c, d) for a, b, c, d in zip(op.v, op.w, op.re, op.im)}


@pytest.mark.parametrize("kind", ["real", "complex"])
def test_commutator_equals_single_word_oracle(kind):
    n = 40
    Ha = I.random_sum(1, n, 25, kind=kind, max_support=4)
    Oa = I.random_sum(2, n, 300, kind=kind, max_support=8)
    got = mw.commutator(_terms(Ha), _terms(Oa))
    want = _as_dict(orc.commutator(orc.Op(n, *Ha), orc.Op(n, *Oa)))
    assert got.keys() == want.keys()
    assert all(got[k] == want[k] for k in want)  # bit for bit


def test_rk4_step_equals_single_word_oracle():
    n = 10
    Ha = I.tilted_ising_chain(n).arrays()
    O = {k: c for k, c in _terms(I.single(n, "Z", 1).arrays())}
    ref = orc.Op(n, *I.single(n, "Z", 1).arrays())
    for _ in range(4):
        O = mw.rk4_step(_terms(Ha), O, 0.05, max_weight=6, cutoff=1e-10, top_k=300)
        ref = orc.rk4_step(orc.Op(n, *Ha), ref, 0.05, max_weight=6, cutoff=1e-10, top_k=300)
        want = _as_dict(ref)
        assert O.keys() == want.keys() and all(O[k] == want[k] for k in want)
    assert mw.norm(O) == orc.norm(ref)


def _local(key, lo):
    return key[0] >> lo, key[1] >> lo


@pytest.mark.parametrize("seed,lo,N", [(0, 61, 128), (1, 61, 128), (2, 61, 128),
                                        (3, 125, 256), (4, 189, 256), (5, 250, 256)])
def test_commutator_across_the_word_boundary_against_dense(seed, lo, N):
    # strings on a 6-site window that straddles a word boundary (sites 62..67 of a 128-site
    # chain, 126..131 and 190..195 of a 256-site chain) or ends on the last site (251..256):
    # the exact commutator from 2^6 x 2^6 matrices on that window, moved back to the global sites
    width = 6
    rng = np.random.default_rng(seed)

    def rand_terms(m):
        terms = {}
        while len(terms) < m:
            v = int(rng.integers(0, 1 << width)) << lo
            w = int(rng.integers(0, 1 << width)) << lo
            terms[(v, w)] = complex(rng.standard_normal(), rng.standard_normal())
        return list(terms.items())

    H, O = rand_terms(6), rand_terms(10)
    got = mw.commutator(H, O)
    if lo % 64 > 58:
        word = lo // 64  # both words of the boundary are used
        lowmask = (1 << (64 * (word + 1))) - 1
        assert any((k[0] | k[1]) >> (64 * (word + 1)) for k in got)
        assert any((k[0] | k[1]) & lowmask for k in got)
    assert all(((k[0] | k[1]) >> N) == 0 for k in got)
    loc = lambda terms: orc.Op(width, [_local(k, lo)[0] for k, _ in terms], [_local(k, lo)[1] for k, _ in terms],  # noqa: E731
                                [c.real for _, c in terms], [c.imag for _, c in terms])
    m = dense.commutator(dense.op_matrix(loc(H), width), dense.op_matrix(loc(O), width))
    want = {(k[0] << lo, k[1] << lo): c for k, c in dense.decompose(m, width).items() if abs(c) > 1e-12}
    assert got.keys() == want.keys()
    for k, c in want.items():
        assert abs(got[k] - c) <= 1e-12 * max(1.0, abs(c))


def test_moving_by_whole_words_moves_the_result():
    n = 12
    Ha = _terms(I.random_sum(5, n, 20, kind="real", max_support=3))
    Oa = _terms(I.random_sum(6, n, 200, kind="real", max_support=6))
    base = mw.commutator(Ha, Oa)
    for s in (64, 100, 130):
        sh = lambda terms: [((k[0] << s, k[1] << s), c) for k, c in terms]  # noqa: E731
        moved = mw.commutator(sh(Ha), sh(Oa))
        assert moved == {(k[0] << s, k[1] << s): c for k, c in base.items()}


def test_product_phase_table_on_far_sites():
    # XY = iZ, YZ = iX, ZX = iY on site 100 (two words away from site 1)
    X = (0, 1 << 99)
    Y = (1 << 99, 1 << 99)
    Z = (1 << 99, 0)
    assert mw.product(X, Y) == (Z, 1)
    assert mw.product(Y, Z) == (X, 1)
    assert mw.product(Z, X) == (Y, 1)
    assert mw.anticommute(X, Y) and not mw.anticommute(X, X)
    # the same on site 256, the last site of a four-word mask
    X, Y, Z = (0, 1 << 255), (1 << 255, 1 << 255), (1 << 255, 0)
    assert mw.product(X, Y) == (Z, 1) and mw.product(Y, Z) == (X, 1) and mw.product(Z, X) == (Y, 1)
    assert mw.product(Y, X) == (Z, 3)


# ----------------------------------------------------------------------------- truncation, RK4 with
# dissipation, Lanczos and trace products (the rest of the path for masks of any width)
def _dict(arrays):
    return dict(_terms(arrays))


def _shift(terms, s):
    return [((k[0] << s, k[1] << s), c) for k, c in terms]


def test_truncate_dissipation_keep_equals_single_word_oracle():
    n = 20
    A = I.random_sum(31, n, 600, kind="complex", max_support=7)
    keep_arr = (A[0][::37], A[1][::37], np.ones(len(A[0][::37])), np.zeros(len(A[0][::37])))
    for kw in (dict(gamma=0.3, dt=0.1), dict(max_weight=5, cutoff=0.05), dict(top_k=150, gamma=0.2, dt=0.05),
               dict(top_k=100, max_weight=6)):
        got = mw.truncate(_dict(A), keep=set(zip(map(int, keep_arr[0]), map(int, keep_arr[1]))), **kw)
        want = _as_dict(orc.truncate(orc.Op(n, *A), keep=orc.Op(n, *keep_arr), **kw))
        assert got.keys() == want.keys() and all(got[k] == want[k] for k in want), kw


def test_rk4_with_dissipation_and_trimmed_stages_equals_single_word_oracle():
    n = 10
    Ha = I.tilted_ising_chain(n).arrays()
    O = _dict(I.single(n, "Z", 1).arrays())
    ref = orc.Op(n, *I.single(n, "Z", 1).arrays())
    for _ in range(5):
        O = mw.rk4_step(_terms(Ha), O, 0.05, top_k=120, gamma=0.1, trim_stages=1)
        ref = orc.rk4_step(orc.Op(n, *Ha), ref, 0.05, top_k=120, gamma=0.1, trim_stages=1)
        want = _as_dict(ref)
        assert O.keys() == want.keys() and all(O[k] == want[k] for k in want)


def test_lanczos_step_equals_single_word_oracle():
    n = 12
    Ha = I.xxz_chain(n, 0.5).arrays()
    prev, cur = {}, _dict(I.uniform_sum(n, "X").arrays())
    rprev, rcur = orc.Op.empty(n), orc.Op(n, *I.uniform_sum(n, "X").arrays())
    b = rb = 0.0
    for _ in range(6):
        b, nxt = mw.lanczos_step(_terms(Ha), prev, cur, b, top_k=400)
        rb, rnxt = orc.lanczos_step(orc.Op(n, *Ha), rprev, rcur, rb, top_k=400)
        prev, cur, rprev, rcur = cur, nxt, rcur, rnxt
        assert b == rb
        want = _as_dict(rcur)
        assert cur.keys() == want.keys() and all(cur[k] == want[k] for k in want)


def test_trace_product_equals_single_word_oracle():
    n = 40
    rng = np.random.default_rng(4)
    v, w = I.random_strings(rng, n, 900)
    A = (v[:600], w[:600], rng.standard_normal(600), rng.standard_normal(600))
    B = (v[300:], w[300:], rng.standard_normal(600) * 1e-5, rng.standard_normal(600))
    assert mw.trace_product(_dict(A), _dict(B)) == orc.trace_product(orc.Op(n, *A), orc.Op(n, *B))


def test_lanczos_printed_example_across_the_word_boundary():
    # the paper's worked example (open XX chain of 10 sites + X on site 4, O_0 = X_1) placed on
    # sites 60..69 of a 128-site chain: both mask words are used, and every printed O_n and
    # the b_n implied by its normalisation are reproduced (letters and signs mapped as in the
    # single-word golden test)
    from test_oracle_pins import _load_golden
    golden = _load_golden("lanczos_xx_defect_n10.txt")
    n, s = 10, 59
    b = I.xx_chain(n)
    b.add(1.0, "X", 4)
    H = _shift(_terms(b.arrays()), s)
    prev, cur, bp = {}, dict(_shift(_terms(I.single(n, "X", 1).arrays()), s)), 0.0
    ops, bs = {1: cur}, []
    for step in range(2, 8):
        bp, nxt = mw.lanczos_step(H, prev, cur, bp, cutoff=1e-10)
        bs.append(bp)
        prev, cur = cur, nxt
        ops[step] = cur
    assert any((k[0] | k[1]) >> 64 for k in ops[7]) and any((k[0] | k[1]) & ((1 << 64) - 1) for k in ops[7])
    letters = {(0, 0): "1", (0, 1): "X", (1, 0): "Z", (1, 1): "Y"}
    relabel = {"1": "1", "X": "X", "Y": "Z", "Z": "Y"}
    for step, printed in golden.items():
        got = {"".join(letters[((k[0] >> (s + i)) & 1, (k[1] >> (s + i)) & 1)] for i in range(n)): c
               for k, c in ops[step].items()}
        want = {"".join(relabel[ch] for ch in p): c * (-1) ** (step - 1) for p, c in printed.items()}
        assert set(got) == set(want), step
        for p in want:
            assert abs(got[p] - want[p]) < 6e-11, (step, p)
    assert np.allclose(bs[:6], [2, 2, 2, 2 * math.sqrt(2), 2 * math.sqrt(3), math.sqrt(50 / 3)], rtol=1e-14)


def test_lanczos_open_xx_chain_of_100_sites_is_constant():
    # closed form: open XX chain from an edge X_1 has b_n = 2 until the Krylov space closes
    n = 100
    H = []
    for j in range(n - 1):
        H.append(((0, (1 << j) | (1 << (j + 1))), 1.0 + 0j))                      # X_j X_{j+1}
        H.append((((1 << j) | (1 << (j + 1)), (1 << j) | (1 << (j + 1))), 1.0 + 0j))  # Y_j Y_{j+1}
    prev, cur, b = {}, {(0, 1): 1.0 + 0j}, 0.0
    for _ in range(12):
        b, nxt = mw.lanczos_step(H, prev, cur, b)
        assert b == 2.0
        prev, cur = cur, nxt
