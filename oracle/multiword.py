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
* truncation (depolarising factor, weight, cutoff, top-k with key ties, keep set) as
  ``truncate``;
* one RK4 step as ``rk4_step`` (k1 = i[H,O], X = O + dt/2 k1, ..., S = k1 + 2k2; S + 2k3;
  S + k4; O + dt/6 S; optional trimmed stages), one Lanczos step as ``lanczos_step``
  (A = [H, O_n] - b_n O_{n-1}, b_{n+1} = ||A||, O_{n+1} = trunc(A / b_{n+1}));
* norms and trace products as exact sums rounded once (fractions).

Parity: pinned by ``tests/test_multiword_oracle.py``: equality, bit for bit, with the
single-word C++ oracle for N <= 64 (commutator, truncation with dissipation and keep set,
RK4 with trimmed stages, Lanczos steps, norm, trace product); dense matrices on local supports
that straddle the word boundary at site 64; invariance under moving a whole operator by a
multiple of 64 sites; the paper's printed Lanczos example placed across the word boundary of
a 128-site chain; the open XX chain of 100 sites (b_n = 2).
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


def truncate(A: dict, max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0, gamma: float = 0.0,
             dt: float = 0.0, keep=None) -> dict:
    """Truncation after a step, in this order: the depolarising factor exp(-(gamma dt) wt)
    on both components (wt = pop(v | w); gamma dt rounded first), the weight filter (drop
    wt > max_weight), exact zeros, the strict cutoff on |c|^2 = re*re + im*im, and top-k by
    |c|^2 with exact ties to the smaller key (v, then w); strings of `keep` (a set of keys)
    are exempt from the top-k step only."""
    x = gamma * dt
    items = []
    for (v, w), c in A.items():
        wt = pop(v | w)
        if gamma != 0.0:
            f = math.exp(-(x * float(wt)))
            c = complex(c.real * f, c.imag * f)
        if max_weight >= 0 and wt > max_weight:
            continue
        if c.real == 0.0 and c.imag == 0.0:
            continue
        q = c.real * c.real + c.imag * c.imag
        if cutoff > 0.0 and q < cutoff * cutoff:
            continue
        items.append(((v, w), c, q))
    if top_k > 0 and len(items) > top_k:
        order = sorted(range(len(items)), key=lambda i: (-items[i][2], items[i][0][0], items[i][0][1]))
        kept = set(order[:top_k])
        if keep:
            kept |= {i for i, t in enumerate(items) if t[0] in keep}
        items = [items[i] for i in sorted(kept)]
    return {k: c for k, c, _ in items}


def rk4_step(H, O: dict, dt: float, max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0,
             gamma: float = 0.0, trim_stages: int = 0, keep=None) -> dict:
    """One RK4 step of dO/dt = i[H, O], then truncation (H: list of ((v, w), c)); with
    trim_stages each k_j is cut to its top_k strings right after its commutator."""
    h2, h6 = dt / 2.0, dt / 6.0

    def L(X):
        k = times_i(commutator(H, list(X.items())))
        if trim_stages and top_k > 0:
            k = truncate(k, top_k=top_k)
        return k

    k1 = L(O)
    k2 = L(axpy(O, h2, k1))
    k3 = L(axpy(O, h2, k2))
    k4 = L(axpy(O, dt, k3))
    S = axpy(axpy(axpy(k1, 2.0, k2), 2.0, k3), 1.0, k4)
    return truncate(axpy(O, h6, S), max_weight=max_weight, cutoff=cutoff, top_k=top_k, gamma=gamma, dt=dt,
                    keep=keep)


def divide(A: dict, b: float) -> dict:
    """A / b per component (IEEE division), the normalisation of the Lanczos recursion."""
    return {k: complex(c.real / b, c.imag / b) for k, c in A.items()}


def lanczos_step(H, O_prev: dict, O_cur: dict, b_prev: float, max_weight: int = -1, cutoff: float = 0.0,
                 top_k: int = 0):
    """One step of the recursion of the Krylov section: A = [H, O_cur] - b_prev O_prev,
    b = ||A||, O_next = trunc(A / b).  Returns (b, O_next); (0.0, {}) when b = 0."""
    A = axpy(commutator(H, list(O_cur.items())), -float(b_prev), O_prev)
    b = norm(A)
    if b == 0.0:
        return 0.0, {}
    return b, truncate(divide(A, b), max_weight=max_weight, cutoff=cutoff, top_k=top_k)


def trace_product(A: dict, B: dict) -> complex:
    """Tr(AB)/2^N = sum over strings in both of a_s b_s, each component summed exactly
    (fractions) and rounded once."""
    from fractions import Fraction
    re, im = Fraction(0), Fraction(0)
    for k, a in A.items():
        if k not in B:
            continue
        b = B[k]
        re += Fraction(a.real) * Fraction(b.real) - Fraction(a.imag) * Fraction(b.imag)
        im += Fraction(a.real) * Fraction(b.imag) + Fraction(a.imag) * Fraction(b.real)
    return complex(float(re), float(im))


def norm(A: dict) -> float:
    """sqrt(sum |c|^2) with the sum formed exactly (fractions) and rounded once."""
    from fractions import Fraction
    s = sum((Fraction(c.real) ** 2 + Fraction(c.imag) ** 2 for c in A.values()), Fraction(0))
    return math.sqrt(float(s))
