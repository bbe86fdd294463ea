"""Masks wider than one word (65..256 sites: 2 or 4 words per mask) on the GPU, through the C
ABI, against the multi-word oracle (oracle/multiword.py, pinned to the single-word oracle, to
dense matrices across the word boundary and to the paper's printed Lanczos example).

Small cases compare element by element, bit for bit.  At the full cap (2^20 strings) the
wide path is compared with the single-word path, itself compared with the oracle: a chain of
64 sites placed anywhere inside a 128- or 256-site register (across the word boundary too)
must give the single-word result moved by the same number of sites, bit for bit - a left
shift keeps the order of keys, so even top-k ties resolve the same way."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import multiword as mw
from paper_2410_09654_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2410_09654_gb300 import paulistr as ps  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ps.load(build_if_missing=True)


def _split(x: int, W: int):
    return [(x >> (64 * k)) & ((1 << 64) - 1) for k in range(W)]


def dev(n, terms):
    """Wide device sum from a list/dict of ((v, w), c) with Python-integer masks."""
    items = list(terms.items()) if isinstance(terms, dict) else list(terms)
    W = ps.words_for(n)
    v = np.array([_split(k[0], W) for k, _ in items], np.uint64).reshape(len(items), W)
    w = np.array([_split(k[1], W) for k, _ in items], np.uint64).reshape(len(items), W)
    re = np.array([complex(c).real for _, c in items])
    im = np.array([complex(c).imag for _, c in items])
    return ps.PauliSum.from_arrays(n, v, w, re, im)


def same(gpu: ps.PauliSum, want: dict, what=""):
    got = gpu.to_dict()
    assert got.keys() == want.keys(), f"{what}: string sets differ ({len(got)} vs {len(want)})"
    bad = [k for k in want if got[k] != want[k]]
    assert not bad, f"{what}: {len(bad)} coefficients differ, e.g. {got[bad[0]]} vs {want[bad[0]]}"


def rand_terms(rng, n, m, support, kind="complex", lo=None):
    """m distinct random strings on windows of `support` sites (placed anywhere, or at lo)."""
    out = {}
    while len(out) < m:
        start = int(rng.integers(0, n - support + 1)) if lo is None else lo
        v = int(rng.integers(0, 1 << support)) << start
        w = int(rng.integers(0, 1 << support)) << start
        if v == 0 and w == 0:
            continue
        re = float(rng.standard_normal())
        im = float(rng.standard_normal()) if kind == "complex" else 0.0
        out[(v, w)] = complex(re, im)
    return out


def chain(n, letters_coefs, fields=()):
    """Open chain: sum_j c (A_j B_{j+1}) for each (A, B, c), plus sum_j c A_j for each (A, c)."""
    bits = {"X": (0, 1), "Y": (1, 1), "Z": (1, 0)}
    H = []
    for j in range(n - 1):
        for a, b, c in letters_coefs:
            va, wa = bits[a]
            vb, wb = bits[b]
            H.append((((va << j) | (vb << (j + 1)), (wa << j) | (wb << (j + 1))), complex(c)))
    for j in range(n):
        for a, c in fields:
            va, wa = bits[a]
            H.append(((va << j, wa << j), complex(c)))
    return H


@pytest.mark.parametrize("n", [65, 100, 128, 200, 256])
@pytest.mark.parametrize("kind", ["real", "complex"])
def test_commutator_matches_oracle(n, kind):
    rng = np.random.default_rng(n + (kind == "complex"))
    H = rand_terms(rng, n, 40, 4, kind)
    O = rand_terms(rng, n, 1500, 8, kind)
    # strings that straddle every word boundary and touch the last site
    for b in range(64, n, 64):
        H.update(rand_terms(rng, n, 6, 4, kind, lo=min(b - 2, n - 4)))
        O.update(rand_terms(rng, n, 200, 8, kind, lo=min(b - 4, n - 8)))
    O.update(rand_terms(rng, n, 50, 6, kind, lo=n - 6))
    Hl = list(H.items())
    got = ps.pauli_commutator(dev(n, Hl), dev(n, O))
    same(got, mw.commutator(Hl, list(O.items())), f"[H,O] n={n}")


def test_empty_and_single_operands():
    n = 130
    H = [((1 << 129, 0), 1.0 + 0j)]
    assert len(ps.pauli_commutator(dev(n, H), ps.PauliSum(n))) == 0
    O = {(0, 1 << 129): 0.5 + 0j}  # X on site 130 against Z on site 130
    same(ps.pauli_commutator(dev(n, H), dev(n, O)), mw.commutator(H, list(O.items())), "single")


def test_upload_download_and_rejections():
    n = 100
    rng = np.random.default_rng(3)
    O = rand_terms(rng, n, 3000, 10)
    S = dev(n, O)
    assert len(S) == 3000
    same(S, O, "round trip")
    v, w, re, im = S.download()
    assert v.shape == (3000, 2)
    keys = [(int(a[0]) | (int(a[1]) << 64), int(b[0]) | (int(b[1]) << 64)) for a, b in zip(v, w)]
    assert keys == sorted(keys)  # canonical order: v, then w, as unsigned integers
    with pytest.raises(ps.PauliError):  # a bit at site 101
        dev(n, {(1 << 100, 0): 1.0})
    with pytest.raises(ps.PauliError):  # a repeated string
        ps.PauliSum.from_arrays(n, np.zeros((2, 2), np.uint64), np.ones((2, 2), np.uint64), np.ones(2), np.zeros(2))
    with pytest.raises(ps.PauliError):  # one-word-only entry points refuse wider sums
        ps.pauli_multiply(S, S)
    C = S.copy()
    same(C, O, "copy")


@pytest.mark.parametrize("n", [100, 256])
def test_truncate_matches_oracle(n):
    rng = np.random.default_rng(7)
    O = rand_terms(rng, n, 4000, 9)
    # exact ties of |c| at the top-k boundary: 800 strings share |c|^2 = 9, about the 35th to
    # the 835th largest value, so top 500 and 700 cut through them (ties go to the smaller key)
    for k in list(O)[:800]:
        O[k] = 3.0 + 0j
    keep_keys = list(O)[::97]
    keep = dev(n, {k: 1.0 for k in keep_keys})
    for kw in (dict(max_weight=7), dict(cutoff=0.3), dict(top_k=500), dict(top_k=1000, gamma=0.2),
               dict(top_k=700, max_weight=8, cutoff=0.01)):
        S = dev(n, O)
        ps.pauli_truncate(S, ps.policy(**{k: v for k, v in kw.items() if k != "dt"}), keep=keep, dt=0.05)
        want = mw.truncate(O, keep=set(keep_keys), dt=0.05, **kw)
        same(S, want, f"truncate {kw}")


def test_norm_and_trace_product_exact():
    n = 192
    rng = np.random.default_rng(11)
    A = rand_terms(rng, n, 3000, 12)
    B = dict(list(rand_terms(rng, n, 2000, 12).items()) + [(k, c * 1e-7) for k, c in list(A.items())[:1000]])
    assert ps.pauli_norm(dev(n, A)) == mw.norm(A)
    assert ps.pauli_trace_product(dev(n, A), dev(n, B)) == mw.trace_product(A, B)
    assert ps.pauli_trace_product(dev(n, B), dev(n, A)) == mw.trace_product(A, B)


@pytest.mark.parametrize("n,s", [(100, 58), (256, 188)])
def test_rk4_steps_match_oracle(n, s):
    # tilted Ising chain of 10 sites placed at sites s+1 .. s+10 (across a word boundary)
    H = [((k[0] << s, k[1] << s), c) for k, c in chain(10, [("Z", "Z", 1.0)], [("X", 1.05), ("Z", 0.5)])]
    O = {(1 << (s + 4), 0): 1.0 + 0j}
    G = dev(n, {(1 << (s + 4), 0): 1.0 + 0j})
    Hd = dev(n, H)
    keep_keys = {(1 << (s + 4), 0)}
    keep = dev(n, {k: 1.0 for k in keep_keys})
    for step in range(4):
        ps.pauli_rk4_step(Hd, G, 0.05, ps.policy(top_k=150, gamma=0.1, trim_stages=1), keep=keep)
        O = mw.rk4_step(H, O, 0.05, top_k=150, gamma=0.1, trim_stages=1, keep=keep_keys)
        same(G, O, f"rk4 step {step}")


def test_lanczos_printed_example_across_the_word_boundary():
    # the paper's worked example (XX chain of 10 sites + X_4, O_0 = X_1, cutoff 1e-10) on sites
    # 60..69 of a 128-site register: b_n equal the printed normalisations, O_n the oracle's
    n, s = 128, 59
    H = [((k[0] << s, k[1] << s), c) for k, c in chain(10, [("X", "X", 1.0), ("Y", "Y", 1.0)], [])]
    H.append(((0, 1 << (s + 3)), 1.0 + 0j))
    Hd = dev(n, H)
    prev, cur = ps.PauliSum(n), dev(n, {(0, 1 << s): 1.0 + 0j})
    rprev, rcur = {}, {(0, 1 << s): 1.0 + 0j}
    b = rb = 0.0
    bs = []
    for step in range(6):
        b = ps.pauli_lanczos_step(Hd, prev, cur, b, ps.policy(cutoff=1e-10))
        rb, rn = mw.lanczos_step(H, rprev, rcur, rb, cutoff=1e-10)
        rprev, rcur = rcur, rn
        assert b == rb, step
        same(cur, rcur, f"O_{step + 1}")
        bs.append(b)
    assert np.allclose(bs, [2, 2, 2, 2 * math.sqrt(2), 2 * math.sqrt(3), math.sqrt(50 / 3)], rtol=1e-14)


def test_lanczos_xxz_with_ties_matches_oracle():
    n = 96
    H = chain(n, [("X", "X", 1.0), ("Y", "Y", 1.0), ("Z", "Z", 0.5)])
    O0 = {(0, 1 << j): 1.0 / math.sqrt(n) + 0j for j in range(n)}  # sum X_i, normalised
    Hd = dev(n, H)
    prev, cur = ps.PauliSum(n), dev(n, O0)
    rprev, rcur = {}, dict(O0)
    b = rb = 0.0
    for step in range(4):
        b = ps.pauli_lanczos_step(Hd, prev, cur, b, ps.policy(top_k=600))
        rb, rn = mw.lanczos_step(H, rprev, rcur, rb, top_k=600)
        rprev, rcur = rcur, rn
        assert b == rb, step
        same(cur, rcur, f"O_{step + 1}")


def _shift_arrays(arrs, n_wide, s):
    """Single-word (v, w, re, im) arrays moved up by s sites into (n, W) word arrays."""
    v, w, re, im = arrs
    W = ps.words_for(n_wide)
    vv = np.zeros((len(v), W), np.uint64)
    ww = np.zeros((len(v), W), np.uint64)
    for k in range(W):
        lo = 64 * k - s  # bit 0 of word k holds bit lo of the unshifted mask
        if lo >= 64 or lo <= -64:
            continue
        if lo >= 0:
            vv[:, k] = v >> np.uint64(lo)
            ww[:, k] = w >> np.uint64(lo)
        else:
            vv[:, k] = v << np.uint64(-lo)
            ww[:, k] = w << np.uint64(-lo)
    return vv, ww, re, im


@pytest.mark.parametrize("n_wide,s", [(128, 0), (128, 32), (128, 64), (256, 150)])
def test_full_cap_lanczos_step_equals_single_word_path_moved(n_wide, s):
    # the XXZ chain of 64 sites, O_0 = sum X_i / 8, top 2^20: ramp on the single-word path to
    # the cap, then one step on both paths from the same (moved) state
    n, cap = 64, 1 << 20
    H1 = ps.PauliSum.from_arrays(n, *I.xxz_chain(n, 0.5).arrays())
    prev, cur = ps.PauliSum(n), ps.PauliSum.from_arrays(n, *I.uniform_sum(n, "X").arrays())
    pol = ps.policy(top_k=cap)
    b = 0.0
    for _ in range(30):
        b = ps.pauli_lanczos_step(H1, prev, cur, b, pol)
        if len(cur) >= cap:
            break
    assert len(cur) == cap
    Hw = ps.PauliSum.from_arrays(n_wide, *_shift_arrays(I.xxz_chain(n, 0.5).arrays(), n_wide, s))
    pw = ps.PauliSum.from_arrays(n_wide, *_shift_arrays(prev.download(), n_wide, s))
    cw = ps.PauliSum.from_arrays(n_wide, *_shift_arrays(cur.download(), n_wide, s))
    b1 = ps.pauli_lanczos_step(H1, prev, cur, b, pol)
    bw = ps.pauli_lanczos_step(Hw, pw, cw, b, pol)
    assert bw == b1
    want = _shift_arrays(cur.download(), n_wide, s)
    got = cw.download()
    assert len(got[2]) == cap
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
