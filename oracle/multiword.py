"""CPU oracle of the commutator path for masks wider than one 64-bit word (N > 64 sites).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it.

The paper stores each string as bit masks of any length (one bit per site, in as many
machine words as the chain needs); the method itself does not depend on the width.  Here a
mask is a Python integer, so N is unbounded.  The definitions are those of the single-word
oracle (``oracle.cpp``), written out in Python:

* P(v, w) = (-i)^{pop(v & w)} Z^v X^w, Z bit v, X bit w (site j is bit j - 1);
* P_a P_b = i^k P_{a ^ b}, k = pop(v_c & w_c) - pop(v_a & w_a) - pop(v_b & w_b) + 2 pop(w_a & v_b) mod 4
  (eqs. v12, w12, eps12 in the Hermitian basis);
* [P_a, P_b] = 2 i^k P_{a ^ b} when pop(w_a & v_b) + pop(v_a & w_b) is odd, else 0 (eq. eps_com);
* [H, O] by Alg. 1 (H outer loop in its order, O inner, contributions to one output string
  added sequentially in H order, products rounded separately: no fused multiply-add);
* truncation by weight, cutoff and top-k with key ties (smaller (v, w) kept), as ``truncate``;
* one RK4 step as ``rk4_step`` (k1 = i[H,O], X = O + dt/2 k1, ..., S = k1 + 2k2; S + 2k3;
  S + k4; O + dt/6 S), Lanczos as ``lanczos_step``.

Parity: pinned by ``tests/test_multiword_oracle.py`` (equality with the single-word C++
oracle for N <= 64, dense matrices on local supports that straddle the word boundary at
site 64, and invariance under moving a whole operator by a multiple of 64 sites).
"""
from __future__ import annotations

import math


def pop(x: int) -> int:
    return bin(x).count("1")


def product(a, b):
    """P_a P_b = i^k P_c: returns (c, k) for strings a = (v, w), b = (v, w)."""
    va, wa = a
    vb, wb = b
    vc, wc = va ^ vb, wa ^ wb
    k = (pop(vc & wc) - pop(va & wa) - pop(vb & wb) + 2 * pop(wa & vb)) % 4
    return (vc, wc), k


def anticommute(a, b) -> bool:
    return (pop(a[1] & b[0]) + pop(a[0] & b[1])) % 2 == 1


_IK = [complex(1, 0), complex(0, 1), complex(-1, 0), complex(0, -1)]


def _times_ik(c: complex, k: int) -> complex:
    # exact: a rotation of the components by a power of i
    re, im = c.real, c.imag
    return [complex(re, im), complex(-im, re), complex(-re, -im), complex(im, -re)][k % 4]


def _mul(a: complex, b: complex) -> complex:
    # four separately rounded products and two rounded sums (no fused multiply-add)
    rr = a.real * b.real
    ii = a.imag * b.imag
    ri = a.real * b.imag
    ir = a.imag * b.real
    return complex(rr - ii, ri + ir)


def commutator(H, O):
    """[H, O] for lists of ((v, w), c): Alg. 1 with the anticommutation test; returns a dict
    {(v, w): c} of the non-zero results."""
    acc: dict = {}
    for hk, hc in H:
        for ok, oc in O:
            if not anticommute(hk, ok):
                continue
            key, k = product(hk, ok)
            t = _times_ik(_mul(hc, oc), k)
            t = complex(2.0 * t.real, 2.0 * t.imag)
            acc[key] = acc[key] + t if key in acc else t
    return {k: c for k, c in acc.items() if c != 0}


def axpy(A: dict, alpha: complex, B: dict) -> dict:
    """A + alpha B over the union of supports (absent strings are zero), zeros dropped."""
    out = dict(A)
    for k, c in B.items():
        t = _mul(complex(alpha), c)
        out[k] = out[k] + t if k in out else t
    return {k: c for k, c in out.items() if c != 0}


def times_i(A: dict) -> dict:
    return {k: complex(-c.imag, c.real) for k, c in A.items()}


def truncate(A: dict, max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0) -> dict:
    """Weight filter, strict cutoff on |c|^2 = re*re + im*im, top-k by |c|^2 (ties: smaller key)."""
    items = []
    for (v, w), c in A.items():
        if max_weight >= 0 and pop(v | w) > max_weight:
            continue
        q = c.real * c.real + c.imag * c.imag
        if cutoff > 0.0 and q < cutoff * cutoff:
            continue
        items.append(((v, w), c, q))
    if top_k > 0 and len(items) > top_k:
        items.sort(key=lambda t: (-t[2], t[0][0], t[0][1]))
        items = items[:top_k]
    return {k: c for k, c, _ in items}


def rk4_step(H, O: dict, dt: float, max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0) -> dict:
    """One RK4 step of dO/dt = i[H, O], then truncation (H: list of ((v, w), c))."""
    h2, h6 = dt / 2.0, dt / 6.0
    L = lambda X: times_i(commutator(H, list(X.items())))  # noqa: E731
    k1 = L(O)
    k2 = L(axpy(O, h2, k1))
    k3 = L(axpy(O, h2, k2))
    k4 = L(axpy(O, dt, k3))
    S = axpy(axpy(axpy(k1, 2.0, k2), 2.0, k3), 1.0, k4)
    return truncate(axpy(O, h6, S), max_weight=max_weight, cutoff=cutoff, top_k=top_k)


def norm(A: dict) -> float:
    """sqrt(sum |c|^2) with the sum formed exactly (fractions) and rounded once."""
    from fractions import Fraction
    s = sum((Fraction(c.real) ** 2 + Fraction(c.imag) ** 2 for c in A.values()), Fraction(0))
    return math.sqrt(float(s))
