"""Pins of the oracle of the FP32 mode with compensated sums (oracle/f32c.py): Sum2 against
exact sums within its published bound and on a case plain FP32 gets wrong, exactness on
dyadic data, dense commutators within the FP32 bound, the paper's printed Lanczos
coefficients, and the FP64 method within FP32 error.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as orc
from oracle import dense
from oracle import f32c
from paper_2410_09654_gb300 import inputs as I

U = 2.0 ** -24  # unit roundoff of FP32


def op(n, arrays):
    return orc.Op(n, *arrays)


def test_two_sum_is_exact():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        a, b = np.float32(rng.standard_normal() * 2.0 ** rng.integers(-30, 30)), np.float32(rng.standard_normal())
        s, e = f32c.two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))


def test_sum2_recovers_what_plain_fp32_loses():
    t = [np.float32(1.0), np.float32(2.0 ** -30), np.float32(-1.0)]
    assert np.float32(np.float32(t[0] + t[1]) + t[2]) == 0.0  # plain FP32 loses the small term
    assert f32c.sum2(t) == np.float32(2.0 ** -30)             # Sum2 keeps it exactly


@pytest.mark.parametrize("seed", range(5))
def test_sum2_within_its_bound(seed):
    # |Sum2 - s| <= u |s| + gamma_{n-1}^2 sum |t_i|  (Ogita, Rump, Oishi, Prop. 4.5)
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 200))
    t = [np.float32(x) for x in rng.standard_normal(n) * np.exp(rng.uniform(-8, 8, n))]
    t[-1] = np.float32(-float(sum(Fraction(float(x)) for x in t[:-1])))  # heavy cancellation
    exact = sum(Fraction(float(x)) for x in t)
    got = Fraction(float(f32c.sum2(t)))
    g = (n - 1) * U / (1 - (n - 1) * U)
    bound = U * abs(exact) + g * g * sum(abs(Fraction(float(x))) for x in t)
    assert abs(got - exact) <= bound


def test_dyadic_data_is_exact():
    n = 8
    H = op(n, I.random_sum(3, n, 20, kind="real", dyadic=True))
    O = op(n, I.random_sum(4, n, 40, kind="real", dyadic=True))
    a, b = f32c.commutator(H, O), orc.commutator(H, O)
    assert np.array_equal(a.v, b.v) and np.array_equal(a.w, b.w) and np.array_equal(a.re, b.re)
    c, d = f32c.add(O, 0.5, a), orc.axpy(O, 0.5, b)
    assert np.array_equal(c.v, d.v) and np.array_equal(c.re, d.re) and np.array_equal(c.im, d.im)


@pytest.mark.parametrize("kind", ["real", "complex"])
def test_commutator_within_fp32_bound_of_dense(kind):
    n = 4
    H = orc.round32(op(n, I.random_sum(5, n, 12, kind=kind)))
    O = orc.round32(op(n, I.random_sum(6, n, 15, kind=kind)))
    got = f32c.commutator(H, O).to_dict()
    m = dense.commutator(dense.op_matrix(H, n), dense.op_matrix(O, n))
    want = {k: c for k, c in dense.decompose(m, n).items() if abs(c) > 1e-9}
    # every term has relative error <= 3u (complex FP32 product) and Sum2 adds u |s| + O(u^2)
    scale = 2 * max(abs(c) for c in H.re + 1j * H.im) * max(abs(c) for c in O.re + 1j * O.im) * len(H)
    assert set(want) <= set(got)
    for k, c in got.items():
        assert abs(c - want.get(k, 0.0)) <= 4 * U * scale, (k, c, want.get(k))


def test_compensation_matters_on_a_small_case():
    # one string receiving the terms 1, 2^-24 and -1 (three sources of one merge): a plain FP32
    # running sum gives 0, the compensated sum keeps 2^-24
    n = 3
    A = orc.Op(n, [1], [0], [1.0], [0.0])
    B = orc.Op(n, [1], [0], [2.0 ** -24], [0.0])
    got = f32c.merge(sources=[(1.0, A), (1.0, B), (-1.0, A)], n_sites=n)
    assert len(got) == 1 and got.re[0] == 2.0 ** -24


def test_lanczos_reproduces_the_printed_coefficients():
    n = 10
    b = I.xx_chain(n)
    b.add(1.0, "X", 4)
    H = op(n, b.arrays())
    prev, cur, bp = orc.Op.empty(n), op(n, I.single(n, "X", 1).arrays()), 0.0
    bs = []
    for _ in range(6):
        bp, nxt = f32c.lanczos_step(H, prev, cur, bp, cutoff=1e-10)
        prev, cur = cur, nxt
        bs.append(bp)
    want = [2, 2, 2, 2 * math.sqrt(2), 2 * math.sqrt(3), math.sqrt(50 / 3)]
    assert np.allclose(bs, want, rtol=20 * U, atol=0)


def test_rk4_within_fp32_error_of_the_fp64_method():
    n = 8
    H = orc.round32(op(n, I.tilted_ising_chain(n).arrays()))
    O64 = O32 = op(n, I.single(n, "Z", 1).arrays())
    for _ in range(6):
        O64 = orc.rk4_step(H, O64, 0.05, top_k=400, gamma=0.1, trim_stages=1)
        O32 = f32c.rk4_step(H, O32, 0.05, top_k=400, gamma=0.1, trim_stages=1)
    a, b = O32.to_dict(), O64.to_dict()
    diff = math.sqrt(sum(abs(a.get(k, 0) - b.get(k, 0)) ** 2 for k in set(a) | set(b)))
    assert diff <= 1e-5 * orc.norm(O64)
    assert np.array_equal(O32.re, O32.re.astype(np.float32).astype(np.float64))
