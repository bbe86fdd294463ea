"""Pins of the multi-word oracle (oracle/multiword.py, masks of any width): equality with the
single-word C++ oracle for N <= 64, dense matrices on local supports that straddle the word
boundary at site 64, and invariance under moving an operator by whole words.  CPU only."""
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


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_commutator_across_the_word_boundary_against_dense(seed):
    # strings on sites 62..67 of a 128-site chain: both words of a two-word mask; the exact
    # commutator from 2^6 x 2^6 matrices on that window, moved back to the global sites
    lo, width, N = 61, 6, 128
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
    assert any((k[0] | k[1]) >> 64 for k in got) and any((k[0] | k[1]) & ((1 << 64) - 1) for k in got)
    loc = lambda terms: orc.Op(width, [_local(k, lo)[0] for k, _ in terms], [_local(k, lo)[1] for k, _ in terms],  # noqa: E731
                                [c.real for _, c in terms], [c.imag for _, c in terms])
    m = dense.commutator(dense.op_matrix(loc(H), width), dense.op_matrix(loc(O), width))
    want = {(k[0] << lo, k[1] << lo): c for k, c in dense.decompose(m, width).items() if abs(c) > 1e-12}
    assert got.keys() == want.keys()
    for k, c in want.items():
        assert abs(got[k] - c) <= 1e-12 * max(1.0, abs(c))
    assert N > 64


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
