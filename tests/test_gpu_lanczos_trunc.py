"""The Lanczos truncation of a single-component FP64 sum by top-k alone ranks the undivided
values (the rank value |RN(x/b)|^2 is non-decreasing in |x|) and divides only the kept
strings.  Checked against the general path (every candidate divided first) and the oracle,
bit for bit: over Lanczos steps of the XXZ chain, and on a built case where two different
values |x| round to the same rank value and the cut falls between them, so that the key
(not |x|) must decide which one is kept."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import assert_match
from paper_2410_09654_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2410_09654_gb300 import paulistr as ps  # noqa: E402


def _step(H, prev, cur, b, k, general):
    """One Lanczos step from copies of (prev, cur); returns b_n and O_{n+1} (canonical order)."""
    ps.pauli_debug_general_truncation(1 if general else 0)
    try:
        p, c = prev.copy(), cur.copy()
        bn = ps.pauli_lanczos_step(H, p, c, b, ps.policy(top_k=k))
        return bn, c.download()
    finally:
        ps.pauli_debug_general_truncation(0)


def _same(x, y):
    """Bit equality of two GPU results (keys and coefficients, signs of zeros included)."""
    return all(np.array_equal(np.asarray(a).view(np.uint64), np.asarray(c).view(np.uint64)) for a, c in zip(x, y))


def _oracle_step(n, Ha, prev, cur, b, k):
    """The oracle's step from the same state; Ha: H's arrays in their given order (the order of
    Alg. 1's outer loop, which fixes the rounding of every sum)."""
    return orc.lanczos_step(orc.Op(n, *Ha), orc.Op(n, *prev.download()) if len(prev) else orc.Op.empty(n),
                            orc.Op(n, *cur.download()), b, top_k=k)


def test_lanczos_steps_fast_truncation_equals_general_and_oracle():
    n, k = 64, 1 << 12
    Ha = I.xxz_chain(n, 0.5).arrays()
    H = ps.PauliSum.from_arrays(n, *Ha)
    x = I.uniform_sum(n, "X").arrays()
    prev, cur = ps.PauliSum(n), ps.PauliSum.from_arrays(n, x[0], x[1], x[2] / 8, x[3])
    b = 0.0
    for step in range(12):
        bf, of = _step(H, prev, cur, b, k, general=False)
        bg, og = _step(H, prev, cur, b, k, general=True)
        assert bf == bg and _same(of, og), step
        if step in (6, 11):  # at the cap: the oracle from the same state
            bo, oo = _oracle_step(n, Ha, prev, cur, b, k)
            assert bf == bo, step
            assert_match(of, oo, exact=True, what=f"step {step}")
        b = ps.pauli_lanczos_step(H, prev, cur, b, ps.policy(top_k=k))


def test_tie_between_different_values_is_broken_by_key():
    n = 24
    Ha = (np.array([1], np.uint64), np.array([0], np.uint64), np.array([0.5]), np.array([0.0]))
    H = ps.PauliSum.from_arrays(n, *Ha)
    # [0.5 Z_1, c X_1 P] = c (phase) Z_1 X_1 P: A holds the coefficients c up to one common phase
    dense = [0.99]
    for _ in range(399):
        dense.append(np.nextafter(dense[-1], 2.0))
    dense = np.array(dense)                       # consecutive doubles, ascending
    rng = np.random.default_rng(7)
    rest = np.concatenate([np.full(200, 0.98), rng.uniform(0.01, 0.9, 1000)])
    # a filler string sets ||A|| so that the quotients of the dense group sit just above a power
    # of two: there two neighbouring values share one rounded quotient
    target = 0.99 / (2.0 ** -5 * 1.0001)
    filler = np.sqrt(target ** 2 - np.sum(dense ** 2) - np.sum(rest ** 2))
    coef = np.concatenate([dense, rest, [filler]])
    m = len(coef)
    # keys: in the dense group a larger value has a larger key (so a tie keeps the smaller value)
    v = (np.arange(m, dtype=np.uint64) + np.uint64(1)) << np.uint64(1)
    w = np.ones(m, np.uint64)
    cur = ps.PauliSum.from_arrays(n, v, w, coef, np.zeros(m))
    prev = ps.PauliSum(n)
    # b as the step computes it, then the rank values |RN(c/b)|^2 in IEEE arithmetic
    b_n, _ = _step(H, prev, cur, 0.0, m, general=True)
    f = (dense / b_n) ** 2
    d = len(dense)
    pairs = [i for i in range(1, d - 2) if f[i] == f[i + 1] and f[i - 1] != f[i] and f[i + 2] != f[i + 1]]
    assert pairs, "the built case must hold two different values with one rank value"
    i = pairs[len(pairs) // 2]
    # cut so that exactly one of the tied pair is kept: everything above the pair, plus one
    k = int(np.sum(coef > dense[i + 1])) + 1
    bf, of = _step(H, prev, cur, 0.0, k, general=False)
    bg, og = _step(H, prev, cur, 0.0, k, general=True)
    bo, oo = _oracle_step(n, Ha, prev, cur, 0.0, k)
    assert bf == bg == bo
    assert _same(of, og)
    assert_match(of, oo, exact=True, what="tie by key")
    kept_v = set(np.asarray(of[0]).tolist())  # the strings of A are Z_1 x: v ^ 1
    assert int(v[i]) ^ 1 in kept_v and int(v[i + 1]) ^ 1 not in kept_v  # the smaller key wins the tie
