"""Parity of the CUDA path (through the C ABI) with the CPU oracle on seeded inputs.

Sizes: small cases for the edge cases, and workloads whose merge spans many
bin groups (and forces the split path) for the tiles-and-ragged-tail cases."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as orc
from paper_2410_09654_gb300 import inputs as I

from gpu_util import assert_match

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2410_09654_gb300 import paulistr as ps  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ps.load(build_if_missing=True)


def dev(n, arrays):
    return ps.PauliSum.from_arrays(n, *arrays)


def ref(n, arrays):
    return orc.Op(n, *arrays)


# ----------------------------------------------------------------------------- commutator
@pytest.mark.parametrize("kind", ["real", "imag", "complex"])
@pytest.mark.parametrize("n,mh,mo,sup", [(3, 9, 17, None), (10, 29, 500, 5), (32, 60, 3000, 8), (64, 120, 5000, 10),
                                         (64, 40, 20000, None),
                                         # |H| at the bitmap-width and order-mask boundaries:
                                         # 250 (8-word bitmaps), 256 (largest ranked merge),
                                         # 257 (per-term ballot emission, chained merge)
                                         (20, 250, 4000, 6), (16, 256, 3000, 6), (16, 257, 3000, 6)])
def test_commutator_random(kind, n, mh, mo, sup):
    Ha = I.random_sum(1000 + n, n, mh, "real" if kind != "complex" else "complex", max_support=min(3, n))
    Oa = I.random_sum(2000 + n + mo, n, mo, kind, max_support=sup)
    out = ps.pauli_commutator(dev(n, Ha), dev(n, Oa))
    assert_match(out.download(), orc.commutator(ref(n, Ha), ref(n, Oa)), what="commutator")


def test_commutator_dyadic_exact():
    n = 12
    Ha = I.random_sum(5, n, 40, "real", max_support=3, dyadic=True)
    Oa = I.random_sum(6, n, 3000, "real", max_support=6, dyadic=True)
    out = ps.pauli_commutator(dev(n, Ha), dev(n, Oa))
    assert_match(out.download(), orc.commutator(ref(n, Ha), ref(n, Oa)), what="dyadic")


def test_commutator_workload_many_groups():
    # XXZ chain on 64 sites acting on a Lanczos vector of ~1e4 strings: many bins/groups
    n = 64
    H = I.xxz_chain(n).arrays()
    O0 = I.uniform_sum(n, "X").arrays()
    _, On = orc.lanczos(ref(n, H), ref(n, O0), 6)
    Oa = (On.v, On.w, On.re, On.im)
    out = ps.pauli_commutator(dev(n, H), dev(n, Oa))
    st = ps.pauli_last_merge_stats()
    assert st["groups"] > 4
    assert_match(out.download(), orc.commutator(ref(n, H), On), what="xxz")


def test_commutator_dense_anticommuting_forces_split():
    # all-to-all random H on 8 sites: every output key receives many contributions and
    # bins overflow the shared-memory pass, exercising the split path
    n = 8
    Ha = I.random_sum(77, n, 400, "real")
    Oa = I.random_sum(78, n, 3000, "real")
    out = ps.pauli_commutator(dev(n, Ha), dev(n, Oa))
    assert_match(out.download(), orc.commutator(ref(n, Ha), ref(n, Oa)), what="dense")


@pytest.mark.parametrize("n,mh,mo", [(7, 300, 2500), (6, 600, 4000)])
def test_commutator_long_chains(n, mh, mo):
    # few sites, many terms: output strings collect tens to hundreds of contributions,
    # which exercises the register, local-array and selection orderings of a key's chain
    Ha = I.random_sum(90 + n, n, mh, "real")
    Oa = I.random_sum(91 + n, n, mo, "imag")
    out = ps.pauli_commutator(dev(n, Ha), dev(n, Oa))
    assert_match(out.download(), orc.commutator(ref(n, Ha), ref(n, Oa)), what="long chains")


def test_commutator_edges():
    n = 64
    top = np.uint64(1 << 63)
    # site 64 bits, the all-ones string, the identity
    Ha = ([top, 0, np.uint64(~0 & (2**64 - 1))], [0, top, np.uint64(2**64 - 1)], [1.0, 0.5, 0.25], [0.0, 0.0, 0.0])
    Oa = ([top, np.uint64(2**64 - 1), 0, 1], [top, 0, 0, 1], [1.0, -2.0, 3.0, 0.5], [0.0, 1.0, 0.0, 0.0])
    out = ps.pauli_commutator(dev(n, Ha), dev(n, Oa))
    assert_match(out.download(), orc.commutator(ref(n, Ha), ref(n, Oa)), what="edges")
    # empty operands
    e = ps.PauliSum(n)
    assert len(ps.pauli_commutator(e, dev(n, Oa))) == 0
    assert len(ps.pauli_commutator(dev(n, Ha), e)) == 0
    # commuting operands give an empty result ([XXZ, sum Z] = 0)
    H = dev(16, I.xxz_chain(16).arrays())
    assert len(ps.pauli_commutator(H, dev(16, I.uniform_sum(16, "Z", 1.0).arrays()))) == 0


def test_commutator_n1():
    Ha = ([1], [0], [0.7], [0.0])
    Oa = ([0, 1], [1, 1], [1.0, 0.25], [0.0, -0.5])
    out = ps.pauli_commutator(dev(1, Ha), dev(1, Oa))
    assert_match(out.download(), orc.commutator(ref(1, Ha), ref(1, Oa)), what="n1")


# ----------------------------------------------------------------------------- add / truncate
# ----------------------------------------------------------------------------- operator product
@pytest.mark.parametrize("n,ma,mb,sup", [(3, 9, 17, None), (10, 29, 500, 5), (64, 120, 5000, 10),
                                         (16, 256, 3000, 6), (12, 300, 2000, 6)])
def test_multiply_random(n, ma, mb, sup):
    # ranked merge (|A| <= 256) and chained merge (|A| = 300); complex coefficients
    Aa = I.random_sum(3000 + n, n, ma, "complex", max_support=min(3, n))
    Ba = I.random_sum(4000 + n + mb, n, mb, "complex", max_support=sup)
    out = ps.pauli_multiply(dev(n, Aa), dev(n, Ba))
    assert_match(out.download(), orc.product(ref(n, Aa), ref(n, Ba)), what="product")


@pytest.mark.parametrize("ka,kb", [("real", "real"), ("real", "imag"), ("imag", "complex")])
def test_multiply_classes(ka, kb):
    n = 24
    Aa = I.random_sum(71, n, 60, ka, max_support=4)
    Ba = I.random_sum(72, n, 4000, kb, max_support=8)
    out = ps.pauli_multiply(dev(n, Aa), dev(n, Ba))
    assert_match(out.download(), orc.product(ref(n, Aa), ref(n, Ba)), what=f"product {ka}x{kb}")


def test_multiply_identity_coefficient_is_trace_product():
    n = 20
    Aa = I.random_sum(81, n, 50, "complex", dyadic=True, max_support=4)
    Ba = I.random_sum(82, n, 3000, "complex", dyadic=True, max_support=4)
    have = set(zip(Ba[0].tolist(), Ba[1].tolist()))
    add = [i for i in range(len(Aa[0])) if (int(Aa[0][i]), int(Aa[1][i])) not in have][:20]
    Ba = tuple(np.concatenate([x, y[add]]) for x, y in zip(Ba, Aa))  # 20 strings shared with A
    A, B = dev(n, Aa), dev(n, Ba)
    got = ps.pauli_multiply(A, B).download()
    ident = [complex(re, im) for v, w, re, im in zip(*got) if v == 0 and w == 0]
    assert ident and ident[0] == ps.pauli_trace_product(A, B) != 0


def test_multiply_edges():
    n = 8
    empty = ps.PauliSum(n)
    B = dev(n, I.random_sum(91, n, 50, "real"))
    assert len(ps.pauli_multiply(empty, B)) == 0
    assert len(ps.pauli_multiply(B, empty)) == 0
    ident = dev(n, (np.array([0], np.uint64), np.array([0], np.uint64), np.array([1.0]), np.array([0.0])))
    assert_match(ps.pauli_multiply(ident, B).download(), ref(n, B.download()), what="1 B")
    with pytest.raises(ps.PauliError):
        ps.pauli_multiply(B, B, B)  # out aliases an operand


# ----------------------------------------------------------------------------- coefficients / correlators
def _single(n, v, w):
    return orc.Op(n, [v], [w], [1.0], [0.0])


def test_coefficients_random_queries():
    n = 64
    Oa = I.random_sum(111, n, 20000, "complex", max_support=8)
    O = dev(n, Oa)
    rng = np.random.default_rng(5)
    pick = rng.integers(0, 20000, 300)
    corner = np.array([0, 2**64 - 1], dtype=np.uint64)  # identity and the all-ones key
    qv = np.concatenate([Oa[0][pick], rng.integers(0, 2**63, 100, dtype=np.uint64), Oa[0][pick[:50]], corner])
    qw = np.concatenate([Oa[1][pick], rng.integers(0, 2**63, 100, dtype=np.uint64), Oa[1][pick[:50]], corner])
    assert qv.dtype == np.uint64 and qv[-1] == np.uint64(2**64 - 1)
    got = ps.pauli_coefficients(O, qv, qw)
    Or = ref(n, Oa)
    for j in range(len(qv)):  # Tr(O P_q)/2^N from the oracle's exactly rounded trace product
        assert got[j] == orc.trace_product(Or, _single(n, int(qv[j]), int(qw[j]))), j


def test_coefficients_all_ones_key_and_edges():
    n = 64
    ones = np.uint64(2**64 - 1)
    O = dev(n, (np.array([ones, 3], np.uint64), np.array([ones, 5], np.uint64), np.array([0.25, 1.0]),
                np.array([-1.0, 0.0])))
    got = ps.pauli_coefficients(O, [ones, 3, 3, 7], [ones, 5, 5, 7])
    assert list(got) == [0.25 - 1j, 1.0, 1.0, 0.0]
    assert len(ps.pauli_coefficients(O, [], [])) == 0
    with pytest.raises(ps.PauliError):
        ps.pauli_coefficients(dev(8, I.random_sum(1, 8, 5, "real")), [1 << 9], [0])


def test_two_point_correlators_after_rk4():
    # Tr(O(t) Z_j)/2^N for every site j on the N=10 chain after a few RK4 steps
    n = 10
    Ha = I.chaotic_ising_chain(n).arrays()
    O0 = I.single(n, "Z", 1).arrays()
    H, O = dev(n, Ha), dev(n, O0)
    Hr, Or = ref(n, Ha), ref(n, O0)
    pol = ps.policy(max_weight=6, cutoff=1e-10)
    for _ in range(5):
        ps.pauli_rk4_step(H, O, 0.05, pol)
        Or = orc.rk4_step(Hr, Or, 0.05, max_weight=6, cutoff=1e-10)
    qv = np.array([1 << j for j in range(n)], np.uint64)
    got = ps.pauli_coefficients(O, qv, np.zeros(n, np.uint64))
    want = [orc.trace_product(Or, _single(n, 1 << j, 0)) for j in range(n)]
    assert list(got) == want
    assert got[0] != 0 and got[1] != 0


# ----------------------------------------------------------------------------- translation symmetry
def _with_periodic(n, arrays):
    # add strings of short period (period 1, 2 and n/2 when n is even) to a real sum
    v, w, re, im = arrays
    have = set(zip(v.tolist(), w.tolist()))
    m = (1 << n) - 1 if n < 64 else 2**64 - 1
    extra = [(m, 0), (0x5555555555555555 & m, 0xAAAAAAAAAAAAAAAA & m)]
    if n % 2 == 0:
        half = (1 << (n // 2)) - 1
        extra.append((0x3 | (0x3 << (n // 2)), 0x1 | (0x1 << (n // 2))))
    extra = [e for e in extra if e not in have and e != (0, 0)]
    ev = np.array([e[0] for e in extra], np.uint64)
    ew = np.array([e[1] for e in extra], np.uint64)
    return (np.concatenate([v, ev]), np.concatenate([w, ew]), np.concatenate([re, np.linspace(0.5, 1.5, len(extra))]),
            np.concatenate([im, np.zeros(len(extra))]))


@pytest.mark.parametrize("n", [8, 13, 64])
def test_ts_canonicalize_and_expand(n):
    Xa = _with_periodic(n, I.random_sum(700 + n, n, 3000, "real", max_support=5))
    assert_match(ps.pauli_ts_canonicalize(dev(n, Xa)).download(), orc.ts_canonical_merge(ref(n, Xa)),
                 what="canonicalize")
    Ga = _with_periodic(n, I.random_sum(710 + n, n, 200, "real", max_support=4))
    assert_match(ps.pauli_ts_expand(dev(n, Ga)).download(), orc.ts_expand(ref(n, Ga)), what="expand")


@pytest.mark.parametrize("gen,n", [("xxz", 16), ("ising", 24), ("xxz", 64)])
def test_ts_commutator_and_norm(gen, n):
    H0a = (I.xxz_generator(n, 0.5) if gen == "xxz" else I.tilted_ising_generator(n)).arrays()
    O0r = orc.ts_canonical_merge(ref(n, I.random_sum(720 + n, n, 2000, "real", max_support=6)))
    O0a = (O0r.v, O0r.w, O0r.re, O0r.im)
    H0 = dev(n, H0a)  # the generator list as given (its translates form H's list on both sides)
    out = ps.pauli_ts_commutator(H0, dev(n, O0a))
    want = orc.ts_commutator(ref(n, H0a), O0r)
    assert_match(out.download(), want, what="ts commutator")
    assert ps.pauli_ts_norm(out) == math.sqrt(orc.ts_norm2(want))


def test_ts_lanczos_matches_oracle_steps():
    n = 24
    H0a = I.xxz_generator(n, 0.5).arrays()
    H0, H0r = dev(n, H0a), ref(n, H0a)
    x1 = I.single(n, "X", 1).arrays()
    prev, cur = ps.PauliSum(n), dev(n, x1)
    rprev, rcur = orc.Op.empty(n), ref(n, x1)
    b = rb = 0.0
    pol = ps.policy(top_k=3000)
    for step in range(10):
        b = ps.pauli_ts_lanczos_step(H0, prev, cur, b, pol)
        rb, nxt = orc.ts_lanczos_step(H0r, rprev, rcur, rb, top_k=3000)
        rprev, rcur = rcur, nxt
        assert b == rb, (step, b, rb)
        assert_match(cur.download(), rcur, what=f"ts lanczos {step}")


def test_ts_lanczos_b_equal_expanded_chain():
    n = 10
    H0 = dev(n, I.xxz_generator(n, 0.5).arrays())
    O0 = dev(n, I.single(n, "X", 1).arrays())
    Hf, Of = ps.pauli_ts_expand(H0), ps.pauli_ts_expand(O0)
    # normalise both starts in their own norms (b_n are blind to the constant factor)
    b0, bf0 = ps.pauli_ts_norm(O0), math.sqrt(orc.norm2(ref(n, Of.download())))
    arr = lambda r: (r.v, r.w, r.re, r.im)
    O0 = dev(n, arr(orc.divide(ref(n, O0.download()), b0)))
    Of = dev(n, arr(orc.divide(ref(n, Of.download()), bf0)))
    pt, ct, pf, cf = ps.PauliSum(n), O0, ps.PauliSum(n), Of
    bt = bf = 0.0
    for _ in range(8):
        bt = ps.pauli_ts_lanczos_step(H0, pt, ct, bt)
        bf = ps.pauli_lanczos_step(Hf, pf, cf, bf)
        assert abs(bt - bf) <= 1e-12 * bf, (bt, bf)


def test_ts_rejects_complex():
    n = 8
    Xa = I.random_sum(730, n, 50, "complex", max_support=3)
    with pytest.raises(ps.PauliError):
        ps.pauli_ts_canonicalize(dev(n, Xa))


# ----------------------------------------------------------------------------- |H| beyond 256 (chunked H)
def test_lanczos_lattice_8x8_chunked_h():
    # the 8x8 Heisenberg lattice has 336 strings: H goes through the merge in chunks, the
    # partial sums carried between them, and the Lanczos source joins the last chunk
    n = 64
    Ha = I.heisenberg_2d(8, 8).arrays()
    O0 = I.single(n, "Z", 28).arrays()
    H, Hr = dev(n, Ha), ref(n, Ha)
    prev, cur = ps.PauliSum(n), dev(n, O0)
    rprev, rcur = orc.Op.empty(n), ref(n, O0)
    b = rb = 0.0
    pol = ps.policy(top_k=6000)
    for step in range(6):
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
        rb, nxt = orc.lanczos_step(Hr, rprev, rcur, rb, top_k=6000)
        rprev, rcur = rcur, nxt
        assert b == rb, (step, b, rb)
        assert_match(cur.download(), rcur, what=f"8x8 lanczos {step}")


def test_rk4_lattice_8x8_dissipation_trimmed():
    # the 2D RK4 workload's shape: 8x8 Heisenberg, O = Z at (4,4), dt = 0.02, gamma = 0.1,
    # top-k with trimmed stages
    n = 64
    Ha = I.heisenberg_2d(8, 8).arrays()
    O0 = I.single(n, "Z", 28).arrays()
    H, O = dev(n, Ha), dev(n, O0)
    Hr, Or = ref(n, Ha), ref(n, O0)
    pol = ps.policy(top_k=4000, gamma=0.1, trim_stages=1)
    for step in range(4):
        ps.pauli_rk4_step(H, O, 0.02, pol)
        Or = orc.rk4_step(Hr, Or, 0.02, top_k=4000, gamma=0.1, trim_stages=1)
        assert_match(O.download(), Or, what=f"8x8 rk4 {step}")


def test_add():
    n = 20
    A = I.random_sum(31, n, 4000, "complex", max_support=6)
    B = (A[0][:2000], A[1][:2000], -A[2][:2000], A[3][:2000] * 0.5)  # overlap, with cancellations
    B = (np.concatenate([B[0], I.random_sum(32, n, 3000, "complex", max_support=6)[0]]),
         np.concatenate([B[1], I.random_sum(32, n, 3000, "complex", max_support=6)[1]]),
         np.concatenate([B[2], I.random_sum(32, n, 3000, "complex", max_support=6)[2]]),
         np.concatenate([B[3], I.random_sum(32, n, 3000, "complex", max_support=6)[3]]))
    # drop duplicate strings inside B
    keys = list(zip(B[0].tolist(), B[1].tolist()))
    _, first = np.unique(np.array(keys, dtype=np.uint64), axis=0, return_index=True)
    first = np.sort(first)
    B = tuple(x[first] for x in B)
    for alpha in (1.0, -0.37 + 1.25j, 2.0):
        out = ps.pauli_add(dev(n, A), alpha, dev(n, B))
        assert_match(out.download(), orc.axpy(ref(n, A), alpha, ref(n, B)), what=f"add {alpha}")


@pytest.mark.parametrize("ka,kb,alpha", [("real", "real", 1.0), ("real", "real", -0.75), ("imag", "imag", 0.3),
                                         ("imag", "real", 2j), ("real", "imag", -1.5j), ("real", "real", 0.5j),
                                         ("complex", "real", 1.0)])
def test_add_classes(ka, kb, alpha):
    # single-component (structured) and general merges, alpha real, imaginary or mixed class
    n = 24
    A = I.random_sum(41, n, 3000, ka, max_support=5)
    B = I.random_sum(42, n, 3000, kb, max_support=5)
    out = ps.pauli_add(dev(n, A), alpha, dev(n, B))
    assert_match(out.download(), orc.axpy(ref(n, A), alpha, ref(n, B)), what=f"add {ka} {kb} {alpha}")


@pytest.mark.parametrize("case", range(6))
def test_truncate(case):
    rng = np.random.default_rng(500 + case)
    n = 16
    m = 20000
    v, w = I.random_strings(rng, n, m)
    vals = np.array([1.0, -1.0, 0.5, 0.25, 1e-11, 3e-3, -3e-3, 0.0, 0.125])
    re = vals[rng.integers(0, len(vals), m)]
    im = vals[rng.integers(0, len(vals), m)] * (case % 2)
    keep_idx = rng.choice(m, 5, replace=False)
    keep = (v[keep_idx], w[keep_idx], np.ones(5), np.zeros(5)) if case >= 3 else None
    params = [dict(max_weight=6, cutoff=1e-10, top_k=0, gamma=0.0, dt=0.05),
              dict(max_weight=-1, cutoff=0.0, top_k=3700, gamma=0.0, dt=0.05),
              dict(max_weight=12, cutoff=1e-3, top_k=5000, gamma=0.1, dt=0.02),
              dict(max_weight=-1, cutoff=0.0, top_k=2000, gamma=0.0, dt=0.05),
              dict(max_weight=-1, cutoff=0.0, top_k=1, gamma=0.3, dt=0.1),
              dict(max_weight=9, cutoff=2e-3, top_k=100, gamma=0.0, dt=0.0)][case]
    O = dev(n, (v, w, re, im))
    # drop exact zeros on the input side, as a commutator output never holds them
    pol = ps.policy(params["max_weight"], params["cutoff"], params["top_k"], params["gamma"])
    ps.pauli_truncate(O, pol, None if keep is None else dev(n, keep), params["dt"])
    want = orc.truncate(ref(n, (v, w, re, im)), keep=None if keep is None else ref(n, keep), **params)
    assert_match(O.download(), want, what=f"truncate {case}")


def test_truncate_all_ties():
    # every coefficient equal: the top-k is decided by the key order alone
    n = 30
    rng = np.random.default_rng(9)
    v, w = I.random_strings(rng, n, 5000)
    re = np.full(5000, 0.5)
    im = np.zeros(5000)
    O = dev(n, (v, w, re, im))
    ps.pauli_truncate(O, ps.policy(top_k=1234))
    assert_match(O.download(), orc.truncate(ref(n, (v, w, re, im)), top_k=1234), what="ties")


def test_division_matches_ieee():
    # the Lanczos normalisation divides with one multiply, one FMA and an exact midpoint
    # test; it must equal the IEEE quotient bit for bit (numpy's division is IEEE)
    rng = np.random.default_rng(77)
    m = 1 << 22
    x = rng.standard_normal(m) * 2.0 ** rng.integers(-300, 300, m)
    # near-ties: products of b with values that have short mantissas, powers of two, tiny/huge
    x[:4096] = (rng.integers(1, 1 << 20, 4096) * 2.0 ** rng.integers(-40, 40, 4096))
    x[4096:4200] = [5e-324, -5e-324, 1e-310, 0.0, -0.0, 1e308, -1e308, 2.0 ** -1022] * 13
    for b in (3.0, 0.1, 12.847329889893492, 2.0 ** -30 * 1.9999999999999998, -7.5, 1.0, 2.0 ** 600, 1e-300):
        xb = x.copy()
        xb[4200:8296] = xb[:4096] * b  # exact multiples and their neighbourhoods
        t = torch.from_numpy(xb).cuda()
        got = ps.pauli_debug_divide(t, b).cpu().numpy()
        want = xb / b
        same = (got == want) | (np.isnan(got) & np.isnan(want))
        assert same.all() and np.array_equal(np.signbit(got), np.signbit(want)), (b, int((~same).sum()))


# ----------------------------------------------------------------------------- reductions
def test_norm_and_trace_exact():
    rng = np.random.default_rng(21)
    n = 64
    m = 30000
    v, w = I.random_strings(rng, n, m)
    re = rng.standard_normal(m) * 10.0 ** rng.integers(-60, 20, m)
    im = rng.standard_normal(m) * 10.0 ** rng.integers(-60, 20, m)
    A = (v, w, re, im)
    dA = dev(n, A)
    assert ps.pauli_norm(dA) == orc.norm(ref(n, A))
    B = (np.concatenate([v[:20000], v[20000:] ^ np.uint64(1 << 40)]), w, rng.standard_normal(m), -im)
    assert ps.pauli_trace_product(dA, dev(n, B)) == orc.trace_product(ref(n, A), ref(n, B))
    # cancellation to exactly zero
    C = (v[:4], w[:4], np.array([1e20, 1.0, -1e20, -1.0]), np.zeros(4))
    D = (v[:4], w[:4], np.ones(4), np.zeros(4))
    assert ps.pauli_trace_product(dev(n, C), dev(n, D)) == 0
    assert ps.pauli_norm(ps.PauliSum(n)) == 0.0


# ----------------------------------------------------------------------------- RK4
def test_rk4_chain_n10_config_shape():
    # the RK4 workload: N=10 tilted Ising chain, O(0)=Z_1, dt=0.05, weight <= 6 then cutoff 1e-10
    n = 10
    Ha = I.tilted_ising_chain(n).arrays()
    O = dev(n, I.single(n, "Z", 1).arrays())
    Or = ref(n, I.single(n, "Z", 1).arrays())
    H, Hr = dev(n, Ha), ref(n, Ha)
    pol = ps.policy(max_weight=6, cutoff=1e-10)
    Z1 = dev(n, I.single(n, "Z", 1).arrays())
    for step in range(12):
        ps.pauli_rk4_step(H, O, 0.05, pol)
        Or = orc.rk4_step(Hr, Or, 0.05, max_weight=6, cutoff=1e-10)
        assert_match(O.download(), Or, what=f"rk4 step {step}")
        assert ps.pauli_trace_product(O, Z1) == orc.trace_product(Or, ref(n, I.single(n, "Z", 1).arrays()))


def test_rk4_dissipation_topk_keep():
    n = 16
    Ha = I.heisenberg_2d(4, 4).arrays()
    O0 = I.single(n, "Z", 6).arrays()
    H, Hr = dev(n, Ha), ref(n, Ha)
    O, Or = dev(n, O0), ref(n, O0)
    keep, keepr = dev(n, O0), ref(n, O0)
    pol = ps.policy(top_k=300, gamma=0.1)
    for step in range(6):
        ps.pauli_rk4_step(H, O, 0.02, pol, keep)
        Or = orc.rk4_step(Hr, Or, 0.02, top_k=300, gamma=0.1, keep=keepr)
        assert_match(O.download(), Or, what=f"rk4 diss step {step}")


def test_rk4_trim_stages():
    n = 16
    Ha = I.heisenberg_2d(4, 4).arrays()
    O0 = I.single(n, "Z", 6).arrays()
    H, Hr = dev(n, Ha), ref(n, Ha)
    O, Or = dev(n, O0), ref(n, O0)
    pol = ps.policy(top_k=200, gamma=0.1, trim_stages=1)
    for step in range(5):
        ps.pauli_rk4_step(H, O, 0.02, pol)
        Or = orc.rk4_step(Hr, Or, 0.02, top_k=200, gamma=0.1, trim_stages=1)
        assert_match(O.download(), Or, what=f"rk4 trim step {step}")


def test_rk4_trim_stages_dyadic_ties():
    # dyadic data and dt = 1/4 keep every sum exact, so the stage trims meet many exactly tied
    # |c| (their top-k is decided by the keys); a single-component k_j takes the trim from the
    # merge's rank keys
    n = 12
    Ha = I.xx_chain(n).arrays()
    O0 = I.random_sum(77, n, 300, kind="real", dyadic=True)
    H, Hr = dev(n, Ha), ref(n, Ha)
    O, Or = dev(n, O0), ref(n, O0)
    pol = ps.policy(top_k=150, trim_stages=1)
    for step in range(3):
        ps.pauli_rk4_step(H, O, 0.25, pol)
        Or = orc.rk4_step(Hr, Or, 0.25, top_k=150, trim_stages=1)
        assert_match(O.download(), Or, exact=True, what=f"rk4 trim ties step {step}")


def test_rk4_commuting_and_partly_commuting():
    # H commuting with O: every k_j is empty, the final merge holds the pre operand alone and
    # O is returned unchanged; then an O of which only some strings commute with H
    n = 8
    Ha = I.single(n, "Z", 3).arrays()
    O0 = I.single(n, "Z", 3).arrays()
    H, Hr = dev(n, Ha), ref(n, Ha)
    O, Or = dev(n, O0), ref(n, O0)
    ps.pauli_rk4_step(H, O, 0.1, ps.policy(top_k=4))
    Or = orc.rk4_step(Hr, Or, 0.1, top_k=4)
    assert_match(O.download(), Or, exact=True, what="commuting")
    v, w, re, im = I.random_sum(21, n, 60, kind="real", dyadic=True)
    O, Or = dev(n, (v, w, re, im)), ref(n, (v, w, re, im))
    for step in range(2):
        ps.pauli_rk4_step(H, O, 0.25, ps.policy(top_k=40, trim_stages=1))
        Or = orc.rk4_step(Hr, Or, 0.25, top_k=40, trim_stages=1)
        assert_match(O.download(), Or, exact=True, what=f"partly commuting step {step}")


# ----------------------------------------------------------------------------- Lanczos
def test_lanczos_paper_example():
    n = 10
    hb = I.xx_chain(n)
    hb.add(1.0, "X", 4)
    H, Hr = dev(n, hb.arrays()), ref(n, hb.arrays())
    O0 = I.single(n, "X", 1).arrays()
    prev, cur = ps.PauliSum(n), dev(n, O0)
    rprev, rcur = orc.Op.empty(n), ref(n, O0)
    b = rb = 0.0
    pol = ps.policy(cutoff=1e-10)
    for step in range(10):
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
        rb, nxt = orc.lanczos_step(Hr, rprev, rcur, rb, cutoff=1e-10)
        rprev, rcur = rcur, nxt
        assert b == rb
        assert_match(cur.download(), rcur, what=f"lanczos {step}")
        assert_match(prev.download(), rprev, what=f"lanczos prev {step}")


def test_lanczos_xxz64_topk():
    # the Lanczos workload at reduced size: XXZ N=64, O_0 = sum X_i / 8, top-k cap
    n = 64
    Ha = I.xxz_chain(n).arrays()
    O0 = I.uniform_sum(n, "X").arrays()
    H, Hr = dev(n, Ha), ref(n, Ha)
    prev, cur = ps.PauliSum(n), dev(n, O0)
    rprev, rcur = orc.Op.empty(n), ref(n, O0)
    b = rb = 0.0
    pol = ps.policy(top_k=4000)
    for step in range(9):
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
        rb, nxt = orc.lanczos_step(Hr, rprev, rcur, rb, top_k=4000)
        rprev, rcur = rcur, nxt
        assert b == rb, (step, b, rb)
        assert_match(cur.download(), rcur, what=f"xxz lanczos {step}")


def test_lanczos_literal_sum_z_is_exhausted():
    # O_0 = sum Z_i commutes with the XXZ chain: b_1 = 0, the Krylov space is closed
    n = 64
    H = dev(n, I.xxz_chain(n).arrays())
    prev, cur = ps.PauliSum(n), dev(n, I.uniform_sum(n, "Z").arrays())
    b = ps.pauli_lanczos_step(H, prev, cur, 0.0, ps.policy(top_k=1 << 22))
    assert b == 0.0
    assert len(cur) == n and len(prev) == 0  # left unchanged


def test_lanczos_open_xx_closed_form():
    n = 12
    H = dev(n, I.xx_chain(n).arrays())
    prev, cur = ps.PauliSum(n), dev(n, I.single(n, "X", 1).arrays())
    b = 0.0
    bs = []
    for _ in range(n + 1):
        b = ps.pauli_lanczos_step(H, prev, cur, b)
        bs.append(b)
        if b == 0.0:
            break
    assert bs[: n - 1] == [2.0] * (n - 1) and bs[n - 1] == 0.0
