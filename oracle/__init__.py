"""CPU oracle for the binary Pauli-string commutator path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product (the CUDA library and its binding) never imports, links or runs it, and
the two share no code: the oracle takes plain numpy arrays and returns plain
numpy arrays.

The heavy loops live in ``oracle.cpp`` (plain C++, FP64, no FMA contraction),
compiled on first use with the host's g++ into ``oracle/_build/``.  ``dense.py``
holds an independent dense-matrix checker for tiny systems.

Every function cites the passage of the paper it follows; see ``oracle.cpp``
for the arithmetic.  Parity status: all entry points are pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``; ``mlp.py`` (the learned
truncation scorer and truncation by an arbitrary score) by ``tests/test_mlp_oracle.py``;
the FP32-coefficient compositions at the end of this file by ``tests/test_f32_oracle.py``;
``multiword.py`` (masks wider than 64 sites) by ``tests/test_multiword_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.cpp")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.cpp`` into ``oracle/_build/liboracle.so`` (plain g++)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


_U64P = ctypes.POINTER(ctypes.c_uint64)
_F64P = ctypes.POINTER(ctypes.c_double)
_OP = [_U64P, _U64P, _F64P, _F64P, ctypes.c_int64]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        lib.or_result_size.argtypes = [vp]
        lib.or_result_size.restype = ctypes.c_int64
        lib.or_result_copy.argtypes = [vp, _U64P, _U64P, _F64P, _F64P]
        lib.or_result_nscalars.argtypes = [vp]
        lib.or_result_nscalars.restype = ctypes.c_int64
        lib.or_result_scalars.argtypes = [vp, _F64P]
        lib.or_result_free.argtypes = [vp]
        lib.or_string_product.argtypes = [ctypes.c_uint64] * 4 + [_U64P, _U64P]
        lib.or_string_product.restype = ctypes.c_int
        lib.or_anticommute.argtypes = [ctypes.c_uint64] * 4
        lib.or_anticommute.restype = ctypes.c_int
        lib.or_commutator.argtypes = _OP + _OP
        lib.or_commutator.restype = vp
        lib.or_product.argtypes = _OP + _OP
        lib.or_product.restype = vp
        lib.or_ts_expand.argtypes = _OP + [ctypes.c_int]
        lib.or_ts_expand.restype = vp
        lib.or_ts_canonical_merge.argtypes = _OP + [ctypes.c_int]
        lib.or_ts_canonical_merge.restype = vp
        lib.or_ts_canonical.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _U64P, _U64P]
        lib.or_ts_canonical.restype = ctypes.c_int
        lib.or_ts_period.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
        lib.or_ts_period.restype = ctypes.c_int
        lib.or_ts_commutator.argtypes = _OP + _OP + [ctypes.c_int]
        lib.or_ts_commutator.restype = vp
        lib.or_ts_norm2.argtypes = _OP + [ctypes.c_int]
        lib.or_ts_norm2.restype = ctypes.c_double
        lib.or_ts_lanczos_step.argtypes = _OP + _OP + _OP + [ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                                             ctypes.c_int64, ctypes.c_int]
        lib.or_ts_lanczos_step.restype = vp
        lib.or_axpy.argtypes = _OP + [ctypes.c_double, ctypes.c_double] + _OP
        lib.or_axpy.restype = vp
        lib.or_scale.argtypes = _OP + [ctypes.c_double]
        lib.or_scale.restype = vp
        lib.or_divide.argtypes = _OP + [ctypes.c_double]
        lib.or_divide.restype = vp
        lib.or_norm2.argtypes = _OP
        lib.or_norm2.restype = ctypes.c_double
        lib.or_trace_product.argtypes = _OP + _OP + [_F64P, _F64P]
        lib.or_truncate.argtypes = _OP + [ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                          ctypes.c_double, ctypes.c_double, _U64P, _U64P,
                                          ctypes.c_int64]
        lib.or_truncate.restype = vp
        lib.or_rk4_step.argtypes = _OP + _OP + [ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                                _U64P, _U64P, ctypes.c_int64]
        lib.or_rk4_step.restype = vp
        lib.or_lanczos.argtypes = _OP + _OP + [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_int64]
        lib.or_lanczos.restype = vp
        _lib = lib
        return lib


@dataclass
class Op:
    """A Pauli sum as four parallel arrays (v, w, re, im) on ``n_sites`` sites."""
    n_sites: int
    v: np.ndarray
    w: np.ndarray
    re: np.ndarray
    im: np.ndarray

    def __post_init__(self):
        self.v = np.ascontiguousarray(self.v, dtype=np.uint64)
        self.w = np.ascontiguousarray(self.w, dtype=np.uint64)
        self.re = np.ascontiguousarray(self.re, dtype=np.float64)
        self.im = np.ascontiguousarray(self.im, dtype=np.float64)

    def __len__(self):
        return int(self.v.shape[0])

    @staticmethod
    def empty(n_sites: int) -> "Op":
        z = np.zeros(0)
        return Op(n_sites, z, z, z, z)

    def to_dict(self) -> dict:
        return {(int(a), int(b)): complex(c, d)
                for a, b, c, d in zip(self.v, self.w, self.re, self.im)}

    @staticmethod
    def from_dict(n_sites: int, d: dict) -> "Op":
        keys = sorted(d)
        return Op(n_sites, [k[0] for k in keys], [k[1] for k in keys],
                  [d[k].real for k in keys], [d[k].imag for k in keys])

    def _args(self):
        return [self.v.ctypes.data_as(_U64P), self.w.ctypes.data_as(_U64P),
                self.re.ctypes.data_as(_F64P), self.im.ctypes.data_as(_F64P),
                ctypes.c_int64(len(self))]


def _take(lib, handle, n_sites) -> tuple[Op, np.ndarray]:
    try:
        n = lib.or_result_size(handle)
        v = np.empty(n, np.uint64)
        w = np.empty(n, np.uint64)
        re = np.empty(n, np.float64)
        im = np.empty(n, np.float64)
        if n:
            lib.or_result_copy(handle, v.ctypes.data_as(_U64P), w.ctypes.data_as(_U64P),
                               re.ctypes.data_as(_F64P), im.ctypes.data_as(_F64P))
        ns = lib.or_result_nscalars(handle)
        s = np.empty(ns, np.float64)
        if ns:
            lib.or_result_scalars(handle, s.ctypes.data_as(_F64P))
        return Op(n_sites, v, w, re, im), s
    finally:
        lib.or_result_free(handle)


def string_product(a: tuple[int, int], b: tuple[int, int]) -> tuple[tuple[int, int], int]:
    """P_a P_b = i^k P_c (eqs. v12, w12, eps12 in the Hermitian basis): returns (c, k)."""
    lib = _load()
    vc, wc = ctypes.c_uint64(), ctypes.c_uint64()
    k = lib.or_string_product(a[0], a[1], b[0], b[1], ctypes.byref(vc), ctypes.byref(wc))
    return (vc.value, wc.value), k


def anticommute(a: tuple[int, int], b: tuple[int, int]) -> bool:
    """Eq. eps_com: the commutator of two strings is non-zero iff they anticommute."""
    return bool(_load().or_anticommute(a[0], a[1], b[0], b[1]))


def commutator(H: Op, O: Op) -> Op:
    """[H, O] by Alg. 1 adapted with eq. eps_com (H outer loop in the given order)."""
    lib = _load()
    return _take(lib, lib.or_commutator(*H._args(), *O._args()), O.n_sites)[0]


def product(A: Op, B: Op) -> Op:
    """A B by Alg. 1 proper: every pair, P_a P_b = i^k P_{a^b} (A outer loop in the given order)."""
    lib = _load()
    return _take(lib, lib.or_product(*A._args(), *B._args()), A.n_sites)[0]


# ------------------------------------------------------------------ translation symmetry
# A translation-symmetric operator on a periodic chain of n = n_sites sites is stored as its
# generator O_0 (one representative string per translation orbit): O = sum_{i<n} T_i(O_0).

def ts_canonical(s: tuple[int, int], n: int) -> tuple[tuple[int, int], int]:
    """Orbit representative of s (smallest translate, v then w) and the smallest shift to it."""
    cv, cw = ctypes.c_uint64(), ctypes.c_uint64()
    r = _load().or_ts_canonical(s[0], s[1], n, ctypes.byref(cv), ctypes.byref(cw))
    return (cv.value, cw.value), r


def ts_period(s: tuple[int, int], n: int) -> int:
    return int(_load().or_ts_period(s[0], s[1], n))


def ts_expand(G: Op) -> Op:
    """sum_{k<n} T_k(G) as a plain sum."""
    lib = _load()
    return _take(lib, lib.or_ts_expand(*G._args(), G.n_sites), G.n_sites)[0]


def ts_canonical_merge(X: Op) -> Op:
    """Every string moved to its orbit representative, contributions added by increasing shift."""
    lib = _load()
    return _take(lib, lib.or_ts_canonical_merge(*X._args(), X.n_sites), X.n_sites)[0]


def ts_commutator(H0: Op, O0: Op) -> Op:
    """Generator of [H, O] for translation-symmetric H, O (Alg. 2's sums, representative order)."""
    lib = _load()
    return _take(lib, lib.or_ts_commutator(*H0._args(), *O0._args(), O0.n_sites), O0.n_sites)[0]


def ts_norm2(O0: Op) -> float:
    """||O||^2 / n, exact then rounded once."""
    return float(_load().or_ts_norm2(*O0._args(), O0.n_sites))


def ts_lanczos_step(H0: Op, O_prev: Op, O_cur: Op, b_prev: float, max_weight: int = -1, cutoff: float = 0.0,
                    top_k: int = 0) -> tuple[float, Op]:
    lib = _load()
    h = lib.or_ts_lanczos_step(*H0._args(), *O_prev._args(), *O_cur._args(), float(b_prev), max_weight,
                               float(cutoff), int(top_k), O_cur.n_sites)
    out, sc = _take(lib, h, O_cur.n_sites)
    return float(sc[0]), out


def axpy(A: Op, alpha: complex, B: Op) -> Op:
    """A + alpha*B over the union of supports (listing: ``O + ...``, ``A - b*O0``)."""
    lib = _load()
    alpha = complex(alpha)
    return _take(lib, lib.or_axpy(*A._args(), alpha.real, alpha.imag, *B._args()), A.n_sites)[0]


def scale(A: Op, s: float) -> Op:
    lib = _load()
    return _take(lib, lib.or_scale(*A._args(), float(s)), A.n_sites)[0]


def divide(A: Op, b: float) -> Op:
    """A / b per component (Lanczos listing: ``O = A/b``)."""
    lib = _load()
    return _take(lib, lib.or_divide(*A._args(), float(b)), A.n_sites)[0]


def norm2(A: Op) -> float:
    """sum |c|^2, exact then rounded once (||O||^2 of the Krylov section, read as Tr(O^dag O)/2^N)."""
    return float(_load().or_norm2(*A._args()))


def norm(A: Op) -> float:
    """||O|| = sqrt(Tr(O^dag O)/2^N) = sqrt(sum |c|^2) (Krylov section, ``norm_lanczos``)."""
    return float(np.sqrt(norm2(A)))


def trace_product(A: Op, B: Op) -> complex:
    """Tr(AB)/2^N = sum over common strings of A_s B_s, exact then rounded (eq. correlator)."""
    lib = _load()
    re, im = ctypes.c_double(), ctypes.c_double()
    lib.or_trace_product(*A._args(), *B._args(), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def _keep_args(keep: Op | None):
    if keep is None or len(keep) == 0:
        z = np.zeros(1, np.uint64)
        return [z.ctypes.data_as(_U64P), z.ctypes.data_as(_U64P), ctypes.c_int64(0)], z
    return [keep.v.ctypes.data_as(_U64P), keep.w.ctypes.data_as(_U64P),
            ctypes.c_int64(len(keep))], keep


def truncate(O: Op, max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0,
             gamma: float = 0.0, dt: float = 0.0, keep: Op | None = None) -> Op:
    """Dissipation e^{-gamma dt wt}, weight filter, |c| cutoff, top-k (``add_noise``, ``trim``, ``cutoff``)."""
    lib = _load()
    ka, _hold = _keep_args(keep)
    return _take(lib, lib.or_truncate(*O._args(), int(max_weight), float(cutoff), int(top_k),
                                      float(gamma), float(dt), *ka), O.n_sites)[0]


def rk4_step(H: Op, O: Op, dt: float, max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0,
             gamma: float = 0.0, trim_stages: int = 0, keep: Op | None = None) -> Op:
    """One RK4 step of dO/dt = i[H,O] followed by truncation (Heisenberg time evolution section)."""
    lib = _load()
    ka, _hold = _keep_args(keep)
    return _take(lib, lib.or_rk4_step(*H._args(), *O._args(), float(dt), int(max_weight),
                                      float(cutoff), int(top_k), float(gamma), int(trim_stages),
                                      *ka), O.n_sites)[0]


def lanczos(H: Op, O0: Op, n_steps: int, max_weight: int = -1, cutoff: float = 0.0,
            top_k: int = 0) -> tuple[np.ndarray, Op]:
    """Lanczos recursion of the Krylov section: returns (b_1..b_n, last O_n)."""
    lib = _load()
    op, b = _take(lib, lib.or_lanczos(*H._args(), *O0._args(), int(n_steps), int(max_weight),
                                      float(cutoff), int(top_k)), O0.n_sites)
    return b, op


def lanczos_step(H: Op, O_prev: Op, O_cur: Op, b_prev: float, max_weight: int = -1,
                 cutoff: float = 0.0, top_k: int = 0) -> tuple[float, Op]:
    """One recursion step: A = [H,O_cur] - b_prev O_prev, b = ||A||, O_next = trunc(A/b)."""
    A = axpy(commutator(H, O_cur), -float(b_prev), O_prev)
    b = norm(A)
    if b == 0.0:
        return 0.0, Op.empty(O_cur.n_sites)
    return b, truncate(divide(A, b), max_weight=max_weight, cutoff=cutoff, top_k=top_k)


# ------------------------------------------------------------------ FP32 coefficients
# Precision mode of the benchmark's FP32 pattern: every stored coefficient is an FP32 number.
# A merge forms each output from the exact products of its FP32 inputs (24-bit significands
# multiply exactly in FP64), accumulated in FP64 in the same order as the FP64 path, and
# rounds the result once to FP32 (round to nearest even); outputs that round to zero are
# dropped like exact zeros.  Norms, traces and b_n stay FP64 (exact sums of the FP32 values).
# These functions compose the pinned FP64 entry points above with that rounding, at the
# points where the method stores a result.

def round32(A: Op) -> Op:
    """Every coefficient rounded to the nearest FP32 number; strings that become zero dropped."""
    re = A.re.astype(np.float32).astype(np.float64)
    im = A.im.astype(np.float32).astype(np.float64)
    nz = (re != 0.0) | (im != 0.0)
    return Op(A.n_sites, A.v[nz], A.w[nz], re[nz], im[nz])


def times_i(A: Op) -> Op:
    """i A (exact: a swap of the components and one sign)."""
    return Op(A.n_sites, A.v, A.w, -A.im, A.re.copy())


def truncate_f32(O: Op, max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0, gamma: float = 0.0,
                 dt: float = 0.0, keep: Op | None = None, divisor: float | None = None) -> Op:
    """Truncation of an FP32 sum: the division (Lanczos) and the dissipation factor are applied
    in FP64 and rounded to FP32 before the weight, cutoff and top-k decisions."""
    X = O if divisor is None else divide(O, divisor)
    if gamma != 0.0:
        import math
        f = np.array([math.exp(-((gamma * dt) * float(k))) for k in range(65)])
        wt = np.array([bin(int(a) | int(b)).count("1") for a, b in zip(X.v, X.w)], np.int64)
        X = Op(X.n_sites, X.v, X.w, X.re * f[wt], X.im * f[wt])
    return truncate(round32(X), max_weight=max_weight, cutoff=cutoff, top_k=top_k, keep=keep)


def commutator_f32(H: Op, O: Op) -> Op:
    return round32(commutator(H, O))


def rk4_step_f32(H: Op, O: Op, dt: float, max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0,
                 gamma: float = 0.0, trim_stages: int = 0, keep: Op | None = None) -> Op:
    """The RK4 step of ``rk4_step`` with FP32 coefficients: k_j, the stage inputs and the new
    O are stored in FP32; S = k1 + 2k2 + 2k3 + k4 is formed inside the final merge (FP64)."""
    h2, h6 = dt / 2.0, dt / 6.0

    def L(X):
        k = round32(times_i(commutator(H, X)))
        if trim_stages and top_k > 0:
            k = truncate(k, top_k=top_k)
        return k

    k1 = L(O)
    k2 = L(round32(axpy(O, h2, k1)))
    k3 = L(round32(axpy(O, h2, k2)))
    k4 = L(round32(axpy(O, dt, k3)))
    S = axpy(axpy(axpy(k1, 2.0, k2), 2.0, k3), 1.0, k4)
    On = round32(axpy(O, h6, S))
    return truncate_f32(On, max_weight=max_weight, cutoff=cutoff, top_k=top_k, gamma=gamma, dt=dt, keep=keep)


def lanczos_step_f32(H: Op, O_prev: Op, O_cur: Op, b_prev: float, max_weight: int = -1,
                     cutoff: float = 0.0, top_k: int = 0) -> tuple[float, Op]:
    """``lanczos_step`` with FP32 coefficients: A is stored in FP32, b_n = ||A|| in FP64, and
    O_n = trunc(A / b_n) rounds the quotient to FP32 before truncating."""
    A = round32(axpy(commutator(H, O_cur), -float(b_prev), O_prev))
    b = norm(A)
    if b == 0.0:
        return 0.0, Op.empty(O_cur.n_sites)
    return b, truncate_f32(A, max_weight=max_weight, cutoff=cutoff, top_k=top_k, divisor=b)


# ------------------------------------------------------------------ batched instances
def batch_rk4_step(H_list, O_list, dt: float, caps, trim_stages: int = 0):
    """Independent instances (disorder realisations): ``rk4_step`` of each (H_b, O_b) with its
    own cap as top_k (cap <= 0: none).  The batched CUDA path must equal this instance by
    instance; the instance tag bits it adds to the keys are removed before comparing."""
    return [rk4_step(H, O, dt, top_k=max(int(c), 0), trim_stages=trim_stages)
            for H, O, c in zip(H_list, O_list, caps)]
