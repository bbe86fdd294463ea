"""Pins of the FP32-coefficient compositions of the oracle (end of oracle/__init__.py):
the exact result rounded to FP32 (dense matrices), exactness on dyadic data, the paper's
printed Lanczos coefficients, and the FP32 error bound against the FP64 method.  CPU only."""
import math

import numpy as np
import pytest

import oracle as orc
from oracle import dense
from paper_2410_09654_gb300 import inputs as I

U32 = 2.0 ** -24  # unit roundoff of FP32


def op(n, arrays):
    return orc.Op(n, *arrays)


def _is_f32(x):
    return np.array_equal(x, x.astype(np.float32).astype(np.float64))


def test_round32_values_idempotence_and_zero_drop():
    A = orc.Op(4, [1, 2, 3, 4], [0, 0, 1, 1], [0.1, 1e-50, 3.0, 0.0], [0.0, 0.0, 1.0 / 3.0, 1e-60])
    R = orc.round32(A)
    assert list(R.v) == [1, 3]  # 1e-50 and 1e-60 are below the smallest FP32 subnormal
    assert R.re[0] == float(np.float32(0.1)) and R.im[1] == float(np.float32(1.0 / 3.0))
    assert _is_f32(R.re) and _is_f32(R.im)
    R2 = orc.round32(R)
    assert np.array_equal(R2.re, R.re) and np.array_equal(R2.im, R.im)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_commutator_f32_is_the_exact_commutator_rounded(seed):
    # dense 2^N matrices give the exact commutator (products of FP32 numbers are exact in
    # FP64 and the few terms per string add without loss here); rounding it to FP32 must
    # agree with the FP32 mode to one unit in the last place
    n = 4
    H = orc.round32(op(n, I.random_sum(seed, n, 12, kind="real")))
    O = orc.round32(op(n, I.random_sum(seed + 10, n, 15, kind="real")))
    got = orc.commutator_f32(H, O).to_dict()
    m = dense.commutator(dense.op_matrix(H, n), dense.op_matrix(O, n))
    want = {k: complex(np.complex64(c)) for k, c in dense.decompose(m, n).items() if abs(c) > 1e-12}
    assert set(got) == set(want)
    for k, c in want.items():
        assert abs(got[k] - c) <= 2 * U32 * abs(c), (k, got[k], c)


def test_f32_mode_is_exact_on_dyadic_data():
    n = 8
    H = op(n, I.random_sum(3, n, 20, kind="real", dyadic=True))
    O = op(n, I.random_sum(4, n, 40, kind="real", dyadic=True))
    a, b = orc.commutator_f32(H, O), orc.commutator(H, O)
    assert np.array_equal(a.v, b.v) and np.array_equal(a.re, b.re)
    c, d = orc.round32(orc.axpy(O, 0.5, a)), orc.axpy(O, 0.5, b)
    assert np.array_equal(c.v, d.v) and np.array_equal(c.re, d.re)


def test_lanczos_f32_reproduces_the_printed_coefficients():
    # the paper's worked Lanczos example: b_n = 2, 2, 2, 2 sqrt 2, 2 sqrt 3, sqrt(50/3); with
    # FP32 coefficients and FP64 norms the b_n carry FP32 rounding only
    n = 10
    b = I.xx_chain(n)
    b.add(1.0, "X", 4)
    H = op(n, b.arrays())
    prev, cur, bprev = orc.Op.empty(n), op(n, I.single(n, "X", 1).arrays()), 0.0
    bs = []
    for _ in range(6):
        bprev, nxt = orc.lanczos_step_f32(H, prev, cur, bprev, cutoff=1e-6)
        prev, cur = cur, nxt
        bs.append(bprev)
        assert _is_f32(cur.re) and _is_f32(cur.im)
    want = [2, 2, 2, 2 * math.sqrt(2), 2 * math.sqrt(3), math.sqrt(50 / 3)]
    assert np.allclose(bs, want, rtol=20 * U32, atol=0)


def test_rk4_f32_tracks_fp64_within_fp32_rounding():
    # the FP32 mode stores FP32 numbers and stays within a few hundred FP32 units of the
    # FP64 method over a few steps (each step rounds O, four k_j and three stage inputs)
    n = 8
    H = orc.round32(op(n, I.tilted_ising_chain(n).arrays()))
    O64 = O32 = op(n, I.single(n, "Z", 1).arrays())
    for _ in range(5):
        O64 = orc.rk4_step(H, O64, 0.05, max_weight=6)
        O32 = orc.rk4_step_f32(H, O32, 0.05, max_weight=6)
        assert _is_f32(O32.re) and _is_f32(O32.im)
    a, b = O32.to_dict(), O64.to_dict()
    assert set(a) <= set(b)
    err = math.sqrt(sum(abs(a.get(k, 0) - c) ** 2 for k, c in b.items()))
    assert err <= 500 * U32 * orc.norm(O64), err
    assert err > 0  # FP32 rounding is visible


def test_truncate_f32_rounds_before_deciding():
    # 1 + 2^-30 rounds to 1 in FP32: the cutoff at 1 keeps it only after rounding... and the
    # dissipation product is rounded to FP32 before the cutoff compares it
    n = 3
    O = orc.Op(n, [1, 2], [0, 0], [1.0 - 2.0 ** -30, 0.5], [0.0, 0.0])
    kept = orc.truncate_f32(O, cutoff=1.0)
    assert list(kept.v) == [1] and kept.re[0] == 1.0
    assert len(orc.truncate(O, cutoff=1.0)) == 0
    G = orc.truncate_f32(orc.Op(n, [1], [1], [0.75], [0.0]), gamma=0.1, dt=0.5)
    assert G.re[0] == float(np.float32(0.75 * math.exp(-0.05)))
