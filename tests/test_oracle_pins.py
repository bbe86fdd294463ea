"""Pins for the CPU oracle: each test ties an oracle entry point to something other
than itself (textbook Pauli algebra, dense 2^N matrices, exact rational arithmetic,
closed forms, invariants, or the values the paper prints for its worked example).
Runs without a GPU."""
from __future__ import annotations

import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as orc
from oracle import dense
from paper_2410_09654_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LET = {"I": (0, 0), "X": (0, 1), "Z": (1, 0), "Y": (1, 1)}


def op(n, arrays):
    return orc.Op(n, *arrays)


def as_dict(o):
    return o.to_dict()


def close_dicts(a: dict, b: dict, tol: float):
    keys = set(a) | set(b)
    scale = max([abs(x) for x in list(a.values()) + list(b.values())] + [1e-300])
    for k in keys:
        assert abs(a.get(k, 0) - b.get(k, 0)) <= tol * scale, (k, a.get(k), b.get(k))


# ----------------------------------------------------------------------------- Pauli algebra
# sigma_a sigma_b = delta_ab I + i eps_abc sigma_c (textbook single-site table).
PAULI_TABLE = {
    ("I", "I"): ("I", 1), ("I", "X"): ("X", 1), ("I", "Y"): ("Y", 1), ("I", "Z"): ("Z", 1),
    ("X", "I"): ("X", 1), ("Y", "I"): ("Y", 1), ("Z", "I"): ("Z", 1),
    ("X", "X"): ("I", 1), ("Y", "Y"): ("I", 1), ("Z", "Z"): ("I", 1),
    ("X", "Y"): ("Z", 1j), ("Y", "Z"): ("X", 1j), ("Z", "X"): ("Y", 1j),
    ("Y", "X"): ("Z", -1j), ("Z", "Y"): ("X", -1j), ("X", "Z"): ("Y", -1j),
}


@pytest.mark.parametrize("pair", sorted(PAULI_TABLE))
def test_single_site_pauli_table(pair):
    a, b = pair
    c, k = orc.string_product(LET[a], LET[b])
    want_letter, want_phase = PAULI_TABLE[pair]
    assert c == LET[want_letter]
    assert 1j ** k == want_phase
    # commutator is non-zero exactly for anticommuting (distinct, non-identity) letters
    assert orc.anticommute(LET[a], LET[b]) == (a != b and "I" not in (a, b))


def test_string_product_vs_dense_all_pairs_n3():
    n = 3
    for va, wa, vb, wb in itertools.product(range(8), repeat=4):
        (vc, wc), k = orc.string_product((va, wa), (vb, wb))
        lhs = dense.string_matrix(va, wa, n) @ dense.string_matrix(vb, wb, n)
        rhs = (1j ** k) * dense.string_matrix(vc, wc, n)
        assert np.array_equal(lhs, rhs)


def test_commutator_vs_dense_all_pairs_n2():
    n = 2
    for va, wa, vb, wb in itertools.product(range(4), repeat=4):
        A = orc.Op(n, [va], [wa], [1.0], [0.0])
        B = orc.Op(n, [vb], [wb], [1.0], [0.0])
        got = as_dict(orc.commutator(A, B))
        want = dense.decompose(dense.commutator(dense.op_matrix(A, n), dense.op_matrix(B, n)), n)
        close_dicts(got, want, 0.0)


@pytest.mark.parametrize("kind", ["real", "imag", "complex"])
@pytest.mark.parametrize("n", [3, 4])
def test_commutator_random_sums_vs_dense(kind, n):
    A = op(n, I.random_sum(11 + n, n, 9, kind))
    B = op(n, I.random_sum(23 + n, n, 17, "complex"))
    got = as_dict(orc.commutator(A, B))
    want = dense.decompose(dense.commutator(dense.op_matrix(A, n), dense.op_matrix(B, n)), n)
    close_dicts(got, want, 1e-13)


def test_commutator_xxz_conserves_total_z():
    # U(1): [sum XX+YY+dZZ, sum Z] = 0 exactly (the literal Lanczos workload with O_0 = sum Z_i).
    n = 16
    H = op(n, I.xxz_chain(n).arrays())
    Sz = op(n, I.uniform_sum(n, "Z", 1.0).arrays())
    assert len(orc.commutator(H, Sz)) == 0
    Sx = op(n, I.uniform_sum(n, "X", 1.0).arrays())
    assert len(orc.commutator(H, Sx)) > 0


def test_commutator_dyadic_exact_vs_dense():
    # dyadic coefficients make every sum exact: compare bit for bit
    n = 4
    A = op(n, I.random_sum(5, n, 12, "real", dyadic=True))
    B = op(n, I.random_sum(6, n, 20, "real", dyadic=True))
    got = as_dict(orc.commutator(A, B))
    want = dense.decompose(dense.commutator(dense.op_matrix(A, n), dense.op_matrix(B, n)), n)
    assert set(got) == set(want)
    for k in got:
        assert got[k] == want[k]


# ----------------------------------------------------------------------------- operator product
def test_product_vs_dense_all_pairs_n2():
    # single strings: A B equals the dense matrix product, for every pair of two-site strings
    n = 2
    for va, wa, vb, wb in itertools.product(range(4), repeat=4):
        A = orc.Op(n, [va], [wa], [1.0], [0.0])
        B = orc.Op(n, [vb], [wb], [1.0], [0.0])
        got = as_dict(orc.product(A, B))
        want = dense.decompose(dense.op_matrix(A, n) @ dense.op_matrix(B, n), n)
        close_dicts(got, want, 0.0)


@pytest.mark.parametrize("pair", sorted(PAULI_TABLE))
def test_product_single_site_table(pair):
    a, b = pair
    A = orc.Op(1, [LET[a][0]], [LET[a][1]], [1.0], [0.0])
    B = orc.Op(1, [LET[b][0]], [LET[b][1]], [1.0], [0.0])
    got = as_dict(orc.product(A, B))
    letter, phase = PAULI_TABLE[pair]
    assert got == {LET[letter]: complex(phase)}


@pytest.mark.parametrize("n", [3, 4])
def test_product_random_sums_vs_dense(n):
    A = op(n, I.random_sum(31 + n, n, 11, "complex"))
    B = op(n, I.random_sum(37 + n, n, 19, "complex"))
    got = as_dict(orc.product(A, B))
    want = dense.decompose(dense.op_matrix(A, n) @ dense.op_matrix(B, n), n)
    close_dicts(got, want, 1e-13)


def test_product_minus_reverse_is_commutator_dyadic():
    # AB - BA = [A, B]; with dyadic coefficients every sum is exact, so bit for bit
    n = 5
    A = op(n, I.random_sum(41, n, 14, "real", dyadic=True))
    B = op(n, I.random_sum(42, n, 23, "imag", dyadic=True))
    ab_ba = orc.axpy(orc.product(A, B), -1.0, orc.product(B, A))
    assert as_dict(ab_ba) == as_dict(orc.commutator(A, B))


def test_product_associative_dyadic():
    n = 4
    A = op(n, I.random_sum(51, n, 6, "real", dyadic=True))
    B = op(n, I.random_sum(52, n, 7, "real", dyadic=True))
    C = op(n, I.random_sum(53, n, 5, "imag", dyadic=True))
    assert as_dict(orc.product(orc.product(A, B), C)) == as_dict(orc.product(A, orc.product(B, C)))


def test_product_identity_coefficient_is_trace_product_dyadic():
    # the identity coefficient of A B is Tr(AB)/2^N
    n = 6
    A = op(n, I.random_sum(61, n, 40, "complex", dyadic=True))
    B = op(n, I.random_sum(62, n, 30, "complex", dyadic=True, max_support=3))
    B = orc.axpy(B, 1.0, orc.Op(n, A.v[:10], A.w[:10], A.re[:10], A.im[:10]))  # shared strings
    got = as_dict(orc.product(A, B)).get((0, 0), 0j)
    assert got == orc.trace_product(A, B)
    assert got != 0


# ----------------------------------------------------------------------------- translation symmetry
def _rot(x: int, k: int, n: int) -> int:
    k %= n
    m = (1 << n) - 1
    return ((x << k) | (x >> (n - k))) & m if k else x


def test_ts_canonical_and_period_brute_force():
    rng = np.random.default_rng(3)
    for n in (3, 8, 13, 64):
        for _ in range(200):
            v = int(rng.integers(0, 2**min(n, 62))) & ((1 << n) - 1)
            w = int(rng.integers(0, 2**min(n, 62))) & ((1 << n) - 1)
            if rng.random() < 0.2:  # periodic strings
                d = [x for x in range(1, n + 1) if n % x == 0][int(rng.integers(0, 2))]
                v = sum(((v >> 0) & ((1 << d) - 1)) << (d * j) for j in range(n // d))
                w = sum(((w >> 0) & ((1 << d) - 1)) << (d * j) for j in range(n // d))
            trans = [(_rot(v, k, n), _rot(w, k, n)) for k in range(n)]
            best = min(trans)
            (cv, cw), r = orc.ts_canonical((v, w), n)
            assert (cv, cw) == best and r == trans.index(best)
            assert orc.ts_period((v, w), n) == next(d for d in range(1, n + 1) if trans[d % n] == (v, w))


def _translation_matrix(n: int) -> np.ndarray:
    # U |s_1 ... s_n> = |s_n s_1 ... s_{n-1}>: the value at site j moves to site j + 1 (site 1 is
    # the most significant bit of the basis index, matching dense.string_matrix)
    d = 2 ** n
    U = np.zeros((d, d))
    for b in range(d):
        bits = [(b >> (n - 1 - j)) & 1 for j in range(n)]
        nb = [bits[-1]] + bits[:-1]
        U[sum(x << (n - 1 - j) for j, x in enumerate(nb)), b] = 1.0
    return U


def test_ts_expand_is_sum_of_translates_dense():
    n = 4
    U = _translation_matrix(n)
    G = op(n, I.random_sum(71, n, 6, "complex", max_support=2))
    got = dense.op_matrix(orc.ts_expand(G), n)
    g = dense.op_matrix(G, n)
    want = sum(np.linalg.matrix_power(U, k) @ g @ np.linalg.matrix_power(U, k).T for k in range(n))
    assert np.abs(got - want).max() < 1e-13


def test_ts_commutator_expands_to_full_commutator_dyadic():
    for n in (6, 9):
        H0 = orc.ts_canonical_merge(op(n, I.xxz_generator(n, 0.5).arrays()))
        O0 = orc.ts_canonical_merge(op(n, I.random_sum(80 + n, n, 25, "imag", max_support=4, dyadic=True)))
        lhs = orc.ts_expand(orc.ts_commutator(H0, O0))
        rhs = orc.commutator(orc.ts_expand(H0), orc.ts_expand(O0))
        assert as_dict(lhs) == as_dict(rhs)
        assert len(lhs) > 0


def test_ts_norm_is_full_norm_over_n_dyadic():
    n = 8
    X = I.random_sum(90, n, 30, "complex", max_support=5, dyadic=True)
    # add strings of period 1, 2 and 4
    per = [(0xFF, 0x00), (0x55, 0xAA), (0x11, 0x33)]
    X = tuple(np.concatenate([x, np.array(y)]) for x, y in zip(X, ([p[0] for p in per], [p[1] for p in per],
                                                                    [0.5, -1.0, 2.0], [0.25, 0.0, -0.5])))
    O0 = orc.ts_canonical_merge(op(n, X))
    assert orc.ts_norm2(O0) * n == orc.norm2(orc.ts_expand(O0))


@pytest.mark.parametrize("gen", ["xxz", "ising"])
def test_ts_lanczos_matches_plain_lanczos_of_expanded_chain(gen):
    n = 8
    H0a = (I.xxz_generator(n, 0.5) if gen == "xxz" else I.tilted_ising_generator(n)).arrays()
    H0 = orc.ts_canonical_merge(op(n, H0a))
    O00 = orc.ts_canonical_merge(op(n, I.single(n, "X" if gen == "xxz" else "Z", 1).arrays()))
    # the TS recursion, starting from O_0 normalised in the TS norm
    b0 = math.sqrt(orc.ts_norm2(O00))
    prev, cur, b = orc.Op.empty(n), orc.divide(O00, b0), 0.0
    bs = []
    for _ in range(8):
        b, nxt = orc.ts_lanczos_step(H0, prev, cur, b)
        bs.append(b)
        prev, cur = cur, nxt
    # the plain recursion on the expanded chain, from O_0 normalised in its own norm (the two
    # norms differ by the constant factor n, to which b_n are blind)
    full = orc.ts_expand(O00)
    b_plain, _ = orc.lanczos(orc.ts_expand(H0), orc.divide(full, math.sqrt(orc.norm2(full))), 8)
    assert np.allclose(bs, b_plain, rtol=1e-12, atol=0)
    assert len(set(np.round(bs, 6))) > 2  # a non-trivial sequence


def test_axpy_vs_dense():
    n = 3
    A = op(n, I.random_sum(1, n, 20, "complex"))
    B = op(n, I.random_sum(2, n, 25, "complex"))
    alpha = 0.37 - 1.25j
    got = as_dict(orc.axpy(A, alpha, B))
    want = dense.decompose(dense.op_matrix(A, n) + alpha * dense.op_matrix(B, n), n)
    close_dicts(got, want, 1e-14)
    # A - A vanishes identically (exact zeros are dropped)
    assert len(orc.axpy(A, -1.0, A)) == 0


# ----------------------------------------------------------------------------- exact sums
def _frac_norm2(o):
    return sum(Fraction(float(r)) ** 2 + Fraction(float(i)) ** 2 for r, i in zip(o.re, o.im))


def test_norm2_is_exactly_rounded():
    rng = np.random.default_rng(3)
    m = 400
    v, w = I.random_strings(rng, 64, m)
    re = rng.standard_normal(m) * 10.0 ** rng.integers(-150, 150, m)
    im = rng.standard_normal(m) * 10.0 ** rng.integers(-150, 150, m)
    re[:5] = [5e-324, 1e-310, 2.0 ** -1074, 1.0, 1.0 + 2.0 ** -52]
    o = orc.Op(64, v, w, re, im)
    assert orc.norm2(o) == float(_frac_norm2(o))
    # a sum that a naive left-to-right loop rounds differently
    o2 = orc.Op(64, v[:4], w[:4], [1.0, 2.0 ** -27, 2.0 ** -27, 2.0 ** -27], [0.0] * 4)
    assert orc.norm2(o2) == float(_frac_norm2(o2))


def test_trace_product_is_exactly_rounded_with_cancellation():
    rng = np.random.default_rng(4)
    m = 300
    v, w = I.random_strings(rng, 40, m)
    a_re = rng.standard_normal(m) * 10.0 ** rng.integers(-40, 40, m)
    a_im = rng.standard_normal(m)
    b_re = rng.standard_normal(m)
    b_im = rng.standard_normal(m) * 10.0 ** rng.integers(-40, 40, m)
    A = orc.Op(40, v, w, a_re, a_im)
    # B shares half the strings of A; the other half are new
    B = orc.Op(40, np.concatenate([v[: m // 2], v[m // 2:] ^ np.uint64(1 << 45)]), w, b_re, b_im)
    got = orc.trace_product(A, B)
    fr = Fraction(0)
    fi = Fraction(0)
    bd = {(int(x), int(y)): (Fraction(float(r)), Fraction(float(i)))
          for x, y, r, i in zip(B.v, B.w, B.re, B.im)}
    for x, y, r, i in zip(A.v, A.w, A.re, A.im):
        if (int(x), int(y)) in bd:
            br, bi = bd[(int(x), int(y))]
            r, i = Fraction(float(r)), Fraction(float(i))
            fr += r * br - i * bi
            fi += r * bi + i * br
    assert got.real == float(fr) and got.imag == float(fi)
    # exact cancellation: <A, -A> terms with opposite signs sum to exactly zero
    C = orc.Op(40, np.concatenate([v[:3], v[:3] ^ np.uint64(1 << 50)]), np.concatenate([w[:3], w[:3]]),
               [1e20, 1.0, -1e-20, 1e20, 1.0, -1e-20], [0.0] * 6)
    D = orc.Op(40, C.v, C.w, [1.0, 1.0, 1.0, -1.0, -1.0, -1.0], [0.0] * 6)
    assert orc.trace_product(C, D) == 0


def test_trace_product_is_tr_ab_over_2n():
    n = 3
    A = op(n, I.random_sum(7, n, 15, "complex"))
    B = op(n, I.random_sum(8, n, 15, "complex"))
    want = np.trace(dense.op_matrix(A, n) @ dense.op_matrix(B, n)) / 2 ** n
    assert abs(orc.trace_product(A, B) - want) < 1e-13


# ----------------------------------------------------------------------------- truncation
def _check_truncation(O, out, max_weight, cutoff, top_k, gamma, dt, keep):
    keepset = set() if keep is None else {(int(a), int(b)) for a, b in zip(keep.v, keep.w)}
    cand = {}
    for v, w, re, im in zip(O.v, O.w, O.re, O.im):
        wt = bin(int(v) | int(w)).count("1")
        f = math.exp(-((gamma * dt) * wt)) if gamma else 1.0
        c = complex(re * f, im * f) if gamma else complex(re, im)
        if max_weight >= 0 and wt > max_weight:
            continue
        if c == 0:
            continue
        a2 = c.real * c.real + c.imag * c.imag
        if cutoff > 0 and a2 < cutoff * cutoff:
            continue
        cand[(int(v), int(w))] = (c, a2)
    got = {(int(v), int(w)): complex(re, im) for v, w, re, im in zip(out.v, out.w, out.re, out.im)}
    assert set(got) <= set(cand)
    for k in got:  # dissipated coefficients carried through unchanged
        assert got[k] == cand[k][0]
    if top_k > 0 and len(cand) > top_k:
        order = sorted(cand, key=lambda k: (-cand[k][1], k))
        want = set(order[:top_k]) | (keepset & set(cand))
    else:
        want = set(cand)
    assert set(got) == want
    # property form of the same rule: every kept non-keep string outranks every dropped one
    dropped = set(cand) - set(got)
    kept_ranked = [k for k in got if k not in keepset]
    if dropped and kept_ranked:
        worst_kept = min(kept_ranked, key=lambda k: (cand[k][1], [-x for x in k]))
        best_drop = max(dropped, key=lambda k: (cand[k][1], [-x for x in k]))
        assert (cand[worst_kept][1], [-x for x in worst_kept]) > (cand[best_drop][1], [-x for x in best_drop])


@pytest.mark.parametrize("case", range(6))
def test_truncate_rules(case):
    rng = np.random.default_rng(100 + case)
    n = 12
    m = 400
    v, w = I.random_strings(rng, n, m)
    # coefficients drawn from a small set so that exact |c|^2 ties are frequent
    vals = np.array([1.0, -1.0, 0.5, 0.25, 1e-11, 3e-3, -3e-3, 0.0])
    re = vals[rng.integers(0, len(vals), m)]
    im = vals[rng.integers(0, len(vals), m)] * (case % 2)
    O = orc.Op(n, v, w, re, im)
    keep = orc.Op(n, v[:3], w[:3], [1.0] * 3, [0.0] * 3) if case >= 3 else None
    params = [dict(max_weight=6, cutoff=1e-10, top_k=0, gamma=0.0, dt=0.05),
              dict(max_weight=-1, cutoff=0.0, top_k=37, gamma=0.0, dt=0.05),
              dict(max_weight=8, cutoff=1e-3, top_k=50, gamma=0.1, dt=0.02),
              dict(max_weight=-1, cutoff=0.0, top_k=20, gamma=0.0, dt=0.05),
              dict(max_weight=-1, cutoff=0.0, top_k=1, gamma=0.3, dt=0.1),
              dict(max_weight=5, cutoff=2e-3, top_k=10, gamma=0.0, dt=0.0)][case]
    out = orc.truncate(O, keep=keep, **params)
    _check_truncation(O, out, keep=keep, **params)


def test_truncate_dissipation_matches_exp():
    n = 6
    O = orc.Op(n, [0, 0b11, 0b111111], [1, 0b01, 0b101010], [1.0, 2.0, -1.0], [0.0, 1.0, 0.5])
    out = orc.truncate(O, gamma=0.1, dt=0.02).to_dict()
    for v, w, re, im in zip(O.v, O.w, O.re, O.im):
        wt = bin(int(v) | int(w)).count("1")
        f = math.exp(-0.1 * 0.02 * wt)
        assert abs(out[(int(v), int(w))] - complex(re, im) * f) <= 1e-16


# ----------------------------------------------------------------------------- RK4
def test_rk4_matches_dense_rk4():
    n = 4
    H = op(n, I.tilted_ising_chain(n).arrays())
    O = op(n, I.random_sum(9, n, 30, "real"))
    dt = 0.05
    got = orc.rk4_step(H, O, dt)
    want = dense.decompose(dense.rk4_dense(dense.op_matrix(H, n), dense.op_matrix(O, n), dt), n)
    close_dicts(as_dict(got), want, 1e-13)


def test_rk4_closed_form_single_field():
    # H = h Z_1, O = X_1: O stays in span{X_1, Y_1} with d(x, y)/dt = (2h y, -2h x);
    # RK4 advances (x, y) by the degree-4 Taylor polynomial of dt*A per step.
    h, dt, steps = 0.7, 0.1, 25
    n = 1
    H = orc.Op(n, [1], [0], [h], [0.0])
    O = orc.Op(n, [0], [1], [1.0], [0.0])
    for _ in range(steps):
        O = orc.rk4_step(H, O, dt)
    A = np.array([[0.0, 2 * h], [-2 * h, 0.0]]) * dt
    R = sum(np.linalg.matrix_power(A, k) / math.factorial(k) for k in range(5))
    x, y = np.linalg.matrix_power(R, steps) @ np.array([1.0, 0.0])
    d = O.to_dict()
    assert abs(d.get(LET["X"], 0) - x) < 1e-14 and abs(d.get(LET["Y"], 0) - y) < 1e-14


def test_rk4_converges_to_exact_heisenberg_evolution():
    n = 4
    H = op(n, I.xxz_chain(n, 0.5).arrays())
    Hm = dense.op_matrix(H, n)
    O0 = op(n, I.single(n, "Z", 1).arrays())
    t = 0.4
    errs = []
    for steps in (8, 16):
        O = O0
        for _ in range(steps):
            O = orc.rk4_step(H, O, t / steps)
        exact = dense.decompose(dense.heisenberg_exact(Hm, dense.op_matrix(O0, n), t), n)
        d = as_dict(O)
        errs.append(max(abs(d.get(k, 0) - exact.get(k, 0)) for k in set(d) | set(exact)))
    assert errs[1] < 5e-6
    assert errs[0] / errs[1] > 12  # fourth order: halving dt cuts the error ~16x


def test_rk4_norm_nonincreasing_and_bounded():
    # RK4 on a skew-adjoint generator: |R(iy)|^2 = 1 - y^6/72 + y^8/576 <= 1 for small y
    n = 6
    H = op(n, I.tilted_ising_chain(n).arrays())
    O = op(n, I.single(n, "Z", 3).arrays())
    for _ in range(5):
        O2 = orc.rk4_step(H, O, 0.05)
        assert orc.norm2(O2) <= orc.norm2(O) * (1 + 1e-14)
        assert orc.norm2(O2) >= orc.norm2(O) * (1 - 1e-5)
        O = O2


def test_liouvillian_is_antisymmetric():
    # Re <O, i[H,O]> = 0 for Hermitian H, O (real coefficients): Tr(O i[H,O]) = 0
    n = 10
    H = op(n, I.tilted_ising_chain(n).arrays())
    O = op(n, I.random_sum(12, n, 200, "real", max_support=4))
    k = orc.commutator(H, O)
    k = orc.Op(n, k.v, k.w, -k.im, k.re)  # i * [H, O]
    tp = orc.trace_product(O, k)
    assert abs(tp) <= 1e-13 * orc.norm(O) * orc.norm(k)


def test_dissipation_decreases_norm():
    n = 8
    H = op(n, I.tilted_ising_chain(n).arrays())
    O = op(n, I.single(n, "Z", 1).arrays())
    for _ in range(4):
        O2 = orc.rk4_step(H, O, 0.05, gamma=0.1)
        assert orc.norm2(O2) < orc.norm2(O)
        O = O2


# ----------------------------------------------------------------------------- Lanczos
def test_lanczos_open_xx_from_edge_is_constant():
    # Open XX chain, O_0 = X_1: each step maps one Majorana string to one other, so
    # b_n = 2 for n = 1..N-1 and the Krylov space closes at n = N (b_N = 0).
    for n in (4, 6, 9):
        H = op(n, I.xx_chain(n).arrays())
        O0 = op(n, I.single(n, "X", 1).arrays())
        b, _ = orc.lanczos(H, O0, n + 2)
        assert np.array_equal(b[: n - 1], np.full(n - 1, 2.0))
        assert b[n - 1] == 0.0 and len(b) == n


@pytest.mark.parametrize("model", ["xxz", "tilted"])
def test_lanczos_matches_dense(model):
    n = 4
    H = op(n, (I.xxz_chain(n, 0.5) if model == "xxz" else I.tilted_ising_chain(n)).arrays())
    O0 = op(n, I.single(n, "Z", 2).arrays())
    b, _ = orc.lanczos(H, O0, 8)
    bd = dense.lanczos_dense(dense.op_matrix(H, n), dense.op_matrix(O0, n), 8, n)
    m = min(len(b), len(bd))
    assert m >= 6
    assert np.allclose(b[:m], bd[:m], rtol=1e-10, atol=1e-12)


def _load_golden(name):
    steps = {}
    cur = None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("step"):
                cur = int(line.split()[1])
                steps[cur] = {}
            else:
                re, im, s = line.split()
                steps[cur][s] = complex(float(re), float(im))
    return steps


def test_lanczos_paper_printed_example():
    # The paper prints O_n for n = 0..6 of this run.  Its letters relabel Y and Z
    # relative to the Hermitian basis here, and its Liouvillian has the opposite
    # sign (so O_n differs by (-1)^n): printed "Y" is this basis' Z and vice versa.
    golden = _load_golden("lanczos_xx_defect_n10.txt")
    n = 10
    b = I.xx_chain(n)
    b.add(1.0, "X", 4)
    H = op(n, b.arrays())
    O0 = op(n, I.single(n, "X", 1).arrays())
    relabel = {"1": "1", "X": "X", "Y": "Z", "Z": "Y"}
    prev, cur, bprev = orc.Op.empty(n), O0, 0.0
    ops = {1: O0}
    for step in range(2, 8):
        bprev, nxt = orc.lanczos_step(H, prev, cur, bprev, cutoff=1e-10)
        prev, cur = cur, nxt
        ops[step] = cur
    letters = {(0, 0): "1", (0, 1): "X", (1, 0): "Z", (1, 1): "Y"}
    for step, printed in golden.items():
        o = ops[step]
        got = {"".join(letters[((int(v) >> i) & 1, (int(w) >> i) & 1)] for i in range(n)): complex(re, im)
               for v, w, re, im in zip(o.v, o.w, o.re, o.im)}
        want = {"".join(relabel[ch] for ch in s): c * (-1) ** (step - 1) for s, c in printed.items()}
        assert set(got) == set(want), step
        for s in want:
            assert abs(got[s] - want[s]) < 6e-11, (step, s)
    # the b_n implied by the printed normalisations: 2, 2, 2, 2 sqrt 2, 2 sqrt 3, sqrt(50/3)
    bs, _ = orc.lanczos(H, O0, 6, cutoff=1e-10)
    assert np.allclose(bs, [2, 2, 2, 2 * math.sqrt(2), 2 * math.sqrt(3), math.sqrt(50 / 3)], rtol=1e-14)


def test_lanczos_orthonormal_untruncated():
    n = 5
    H = op(n, I.tilted_ising_chain(n).arrays())
    O = op(n, I.single(n, "Z", 1).arrays())
    prev, cur, b = orc.Op.empty(n), O, 0.0
    basis = [O]
    for _ in range(5):
        b, nxt = orc.lanczos_step(H, prev, cur, b)
        prev, cur = cur, nxt
        basis.append(cur)
    for i, a in enumerate(basis):
        for j, c in enumerate(basis):
            ip = orc.trace_product(orc.Op(n, a.v, a.w, a.re, -a.im), c)  # <a, c> = Tr(a^dag c)/2^N
            assert abs(ip - (1.0 if i == j else 0.0)) < 1e-12
