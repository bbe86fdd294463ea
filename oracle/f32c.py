"""CPU oracle of the FP32 mode with compensated sums (precision PS_COEF_F32C).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it.

Reading of the benchmark's precision pattern ("product coefficients in FP32 and compensated
summation in the merge; FP64 for the Lanczos norms, the b_n recursion and the inner
products"), written as one definition per merge - the unit every step of the method is made
of (Alg. 1 for [H, O]; the linear combinations of the RK4 and Lanczos formulas):

* every input coefficient (H, the operands, the scalars alpha, post) is an FP32 number
  (rounded to nearest FP32 where it is not);
* a product term is 2 i^(k + rot) (h x) with h x the complex product in FP32 arithmetic
  (four rounded products, two rounded sums, exactly-zero products skipped); a source term is
  alpha y in the same arithmetic; the pre operand enters as it is;
* for one output string the terms are added in Alg. 1's order (H index, then the sources in
  formula order) by the compensated sum Sum2 of Ogita, Rump and Oishi (Accurate sum and dot
  product, SIAM J. Sci. Comput. 26, 2005): s_1 = t_1, (s_i, e_i) = TwoSum(s_{i-1}, t_i) with
  Knuth's TwoSum, the errors e_i added in FP32, result RN(s_n + sum e) - per component;
* with a post factor the output is pre + post * acc in FP32 (a zero term is skipped);
* exact zeros are dropped.

The RK4 and Lanczos steps compose merges as the CUDA path does: k_j = i[H, X] (one merge of
products, rot = 1), X = O + c k (one merge of two sources), O' = O + (dt/6)(k1 + 2 k2 + 2 k3 + k4)
(one merge: four sources, pre O, post dt/6); A = [H, O_n] - b_n O_{n-1} (one merge of products and
a source).  Truncation, norms and b_n are those of the FP32 mode (``truncate_f32``, exact FP64
norms).

Parity: pinned by ``tests/test_f32c_oracle.py`` (Sum2 against exact sums within its published
bound and on a case naive FP32 gets wrong, exactness on dyadic data, dense commutators within
the FP32 bound, the paper's printed Lanczos coefficients, the FP64 method within FP32 error).
"""
from __future__ import annotations

import numpy as np

from . import Op, norm, truncate_f32
from .multiword import anticommute, product as string_product

F32 = np.float32


def _f(x) -> np.float32:
    return F32(x)


def two_sum(a: np.float32, b: np.float32):
    """Knuth's TwoSum in FP32: s = RN(a + b) and the exact error e with a + b = s + e."""
    s = F32(a + b)
    z = F32(s - a)
    e = F32(F32(a - F32(s - z)) + F32(b - z))
    return s, e


def sum2(terms) -> np.float32:
    """Sum2 (Ogita, Rump, Oishi) of FP32 numbers in the given order."""
    if not terms:
        return F32(0.0)
    s = F32(terms[0])
    c = F32(0.0)
    for t in terms[1:]:
        s, e = two_sum(s, F32(t))
        c = F32(c + e)
    return F32(s + c)


def _mul(a: np.float32, b: np.float32) -> np.float32:
    return F32(a * b)


def cmul32(a, b):
    """(a.re b.re - a.im b.im, a.re b.im + a.im b.re) in FP32; products with an exactly-zero
    factor skipped (they cannot change a non-zero component)."""
    ar, ai, br, bi = F32(a[0]), F32(a[1]), F32(b[0]), F32(b[1])
    rr = F32(0.0) if ar == 0 or br == 0 else _mul(ar, br)
    ii = F32(0.0) if ai == 0 or bi == 0 else _mul(ai, bi)
    ri = F32(0.0) if ar == 0 or bi == 0 else _mul(ar, bi)
    ir = F32(0.0) if ai == 0 or br == 0 else _mul(ai, br)
    re = rr if ii == 0 else (F32(-ii) if rr == 0 else F32(rr - ii))
    im = ri if ir == 0 else (ir if ri == 0 else F32(ri + ir))
    return re, im


def _rot(c, k):
    re, im = c
    return [(re, im), (F32(-im), re), (F32(-re), F32(-im)), (im, F32(-re))][k % 4]


def _add32(a: np.float32, b: np.float32) -> np.float32:
    if b == 0:
        return a
    if a == 0:
        return b
    return F32(a + b)


def merge(products=None, sources=(), pre: Op | None = None, post=None, n_sites: int | None = None) -> Op:
    """One merge: products = (H, X, rot) or None; sources = [(alpha, Y), ...]; pre and post as
    described in the module docstring.  Returns the FP32-valued result as an Op."""
    terms: dict = {}  # key -> list of (order, (re, im))
    nh = 0
    if products is not None:
        H, X, rot = products
        nh = len(H)
        for hi in range(len(H)):
            hk = (int(H.v[hi]), int(H.w[hi]))
            hc = (_f(H.re[hi]), _f(H.im[hi]))
            for xi in range(len(X)):
                xk = (int(X.v[xi]), int(X.w[xi]))
                if not anticommute(hk, xk):
                    continue
                key, k = string_product(hk, xk)
                p = cmul32(hc, (_f(X.re[xi]), _f(X.im[xi])))
                p = (F32(F32(2.0) * p[0]), F32(F32(2.0) * p[1]))
                terms.setdefault(key, []).append((hi, _rot(p, k + rot)))
    for si, (alpha, Y) in enumerate(sources):
        a = (_f(complex(alpha).real), _f(complex(alpha).imag))
        for yi in range(len(Y)):
            key = (int(Y.v[yi]), int(Y.w[yi]))
            terms.setdefault(key, []).append((nh + si, cmul32(a, (_f(Y.re[yi]), _f(Y.im[yi])))))
    pre_d = {}
    if pre is not None:
        for i in range(len(pre)):
            pre_d[(int(pre.v[i]), int(pre.w[i]))] = (_f(pre.re[i]), _f(pre.im[i]))
    keys = set(terms) | set(pre_d)
    pc = None if post is None else (_f(complex(post).real), _f(complex(post).imag))
    out = {}
    for key in keys:
        lst = sorted(terms.get(key, []), key=lambda t: t[0])
        n = len(lst)
        acc = (sum2([t[1][0] for t in lst]), sum2([t[1][1] for t in lst]))
        if pc is not None:
            sc = cmul32(pc, acc) if n > 0 else (F32(0.0), F32(0.0))
            if key in pre_d:
                pv = pre_d[key]
                r = (_add32(pv[0], sc[0]), _add32(pv[1], sc[1])) if n > 0 else pv
            else:
                r = sc
        else:
            r = acc
        if r[0] != 0 or r[1] != 0:
            out[key] = complex(float(r[0]), float(r[1]))
    if n_sites is None:
        n_sites = (products[1].n_sites if products is not None else
                   (sources[0][1].n_sites if sources else pre.n_sites))
    return Op.from_dict(n_sites, out)


def commutator(H: Op, O: Op) -> Op:
    return merge(products=(H, O, 0))


def add(A: Op, alpha: complex, B: Op) -> Op:
    return merge(sources=[(1.0, A), (alpha, B)], n_sites=A.n_sites)


def rk4_step(H: Op, O: Op, dt: float, max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0,
             gamma: float = 0.0, trim_stages: int = 0, keep: Op | None = None) -> Op:
    h2, h6 = dt / 2.0, dt / 6.0
    n = O.n_sites

    def L(X):
        k = merge(products=(H, X, 1), n_sites=n)
        if trim_stages and top_k > 0:
            k = truncate_f32(k, top_k=top_k)
        return k

    k1 = L(O)
    k2 = L(merge(sources=[(1.0, O), (h2, k1)], n_sites=n))
    k3 = L(merge(sources=[(1.0, O), (h2, k2)], n_sites=n))
    k4 = L(merge(sources=[(1.0, O), (dt, k3)], n_sites=n))
    On = merge(sources=[(1.0, k1), (2.0, k2), (2.0, k3), (1.0, k4)], pre=O, post=h6, n_sites=n)
    return truncate_f32(On, max_weight=max_weight, cutoff=cutoff, top_k=top_k, gamma=gamma, dt=dt, keep=keep)


def lanczos_step(H: Op, O_prev: Op, O_cur: Op, b_prev: float, max_weight: int = -1, cutoff: float = 0.0,
                 top_k: int = 0) -> tuple[float, Op]:
    n = O_cur.n_sites
    src = [(-float(b_prev), O_prev)] if len(O_prev) > 0 else []
    A = merge(products=(H, O_cur, 0), sources=src, n_sites=n)
    b = norm(A)
    if b == 0.0:
        return 0.0, Op.empty(n)
    return b, truncate_f32(A, max_weight=max_weight, cutoff=cutoff, top_k=top_k, divisor=b)
