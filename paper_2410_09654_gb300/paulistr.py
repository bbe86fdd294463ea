"""Thin Python binding of libpaulistr (ctypes).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  The functions carry the names of the C ABI in ``include/paulistr.h``;
``PauliSum`` owns one ``pauli_sum*``.  PyTorch is used only to pick the CUDA
stream (``torch.cuda.current_stream()``) and to pass device tensors.

There is no CPU fallback: if the compiled library is missing, or no CUDA
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

PS_OK = 0
PS_ERR_INVALID = 1
PS_ERR_CAPACITY = 2
PS_ERR_TABLE_FULL = 3
PS_ERR_CUDA = 4
PS_ERR_TIMEOUT = 5
PS_ERR_KRYLOV_EXHAUSTED = 6
PS_ERR_NOMEM = 7
PS_ERR_IO = 9
PS_ERR_NONFINITE = 10
PS_COEF_F64 = 0
PS_COEF_F32 = 1
PS_COEF_F32C = 2

_lib = None


class PauliError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _lib
        msg = lib.pauli_status_string(status).decode() if lib else str(status)
        extra = ""
        if lib and status == PS_ERR_CUDA:
            extra = " [" + lib.pauli_last_cuda_error().decode() + "]"
        super().__init__(f"{where}: {msg}{extra}")
        self.status = status


class pauli_trunc_policy(ctypes.Structure):
    _fields_ = [("max_weight", ctypes.c_int), ("cutoff", ctypes.c_double), ("top_k", ctypes.c_int64),
                ("gamma", ctypes.c_double), ("trim_stages", ctypes.c_int)]


class pauli_merge_stats(ctypes.Structure):
    _fields_ = [("pair_tests", ctypes.c_int64), ("contributions", ctypes.c_int64), ("merged", ctypes.c_int64),
                ("groups", ctypes.c_int64), ("split_groups", ctypes.c_int64)]


def policy(max_weight: int = -1, cutoff: float = 0.0, top_k: int = 0, gamma: float = 0.0,
           trim_stages: int = 0) -> pauli_trunc_policy:
    return pauli_trunc_policy(int(max_weight), float(cutoff), int(top_k), float(gamma), int(trim_stages))


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libpaulistr.so; raise if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libpaulistr is not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    U64P = ctypes.POINTER(ctypes.c_uint64)
    F64P = ctypes.POINTER(ctypes.c_double)
    I64 = ctypes.c_int64
    sig = {
        "pauli_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "pauli_last_cuda_error": ([], ctypes.c_char_p),
        "pauli_sum_create": ([ctypes.c_int, I64, P, ctypes.POINTER(P)], ctypes.c_int),
        "pauli_sum_destroy": ([P], ctypes.c_int),
        "pauli_sum_upload": ([P, U64P, U64P, F64P, F64P, I64], ctypes.c_int),
        "pauli_sum_upload_device": ([P, P, P, P, P, I64], ctypes.c_int),
        "pauli_sum_size": ([P, ctypes.POINTER(I64)], ctypes.c_int),
        "pauli_sum_n_sites": ([P, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "pauli_sum_download": ([P, U64P, U64P, F64P, F64P, I64, ctypes.POINTER(I64)], ctypes.c_int),
        "pauli_sum_download_device": ([P, P, P, P, P, I64, ctypes.POINTER(I64)], ctypes.c_int),
        "pauli_sum_copy": ([P, P], ctypes.c_int),
        "pauli_sum_sort_by_hash": ([P], ctypes.c_int),
        "pauli_sum_save": ([P, ctypes.c_char_p, P, I64], ctypes.c_int),
        "pauli_sum_load": ([P, ctypes.c_char_p, P, I64, ctypes.POINTER(I64)], ctypes.c_int),
        "pauli_commutator": ([P, P, P], ctypes.c_int),
        "pauli_multiply": ([P, P, P], ctypes.c_int),
        "pauli_add": ([P, ctypes.c_double, ctypes.c_double, P, P], ctypes.c_int),
        "pauli_truncate": ([P, ctypes.POINTER(pauli_trunc_policy), P, ctypes.c_double], ctypes.c_int),
        "pauli_rk4_step": ([P, P, ctypes.c_double, ctypes.POINTER(pauli_trunc_policy), P], ctypes.c_int),
        "pauli_lanczos_step": ([P, P, P, ctypes.c_double, ctypes.POINTER(pauli_trunc_policy), F64P], ctypes.c_int),
        "pauli_trace_product": ([P, P, F64P, F64P], ctypes.c_int),
        "pauli_coefficients": ([P, P, P, I64, P, P], ctypes.c_int),
        "pauli_ts_expand": ([P, P], ctypes.c_int),
        "pauli_ts_canonicalize": ([P, P], ctypes.c_int),
        "pauli_ts_commutator": ([P, P, P], ctypes.c_int),
        "pauli_ts_norm": ([P, F64P], ctypes.c_int),
        "pauli_ts_lanczos_step": ([P, P, P, ctypes.c_double, ctypes.POINTER(pauli_trunc_policy), F64P], ctypes.c_int),
        "pauli_norm": ([P, F64P], ctypes.c_int),
        "pauli_last_merge_stats": ([ctypes.POINTER(pauli_merge_stats)], ctypes.c_int),
        "pauli_debug_fail_alloc_after": ([I64], ctypes.c_int),
        "pauli_debug_output_hash": ([P, P, I64, P], ctypes.c_int),
        "pauli_debug_mlp_wait": ([ctypes.c_int, I64], ctypes.c_int),
        "pauli_debug_general_truncation": ([ctypes.c_int], ctypes.c_int),
        "pauli_profile_enable": ([ctypes.c_int], ctypes.c_int),
        "pauli_profile_report": ([ctypes.c_char_p, I64, ctypes.POINTER(I64)], ctypes.c_int),
        "pauli_launch_count": ([], I64),
        "pauli_debug_divide": ([P, I64, ctypes.c_double, P], ctypes.c_int),
        "pauli_trace_product_noalloc": ([P, P, P, P, I64, P, P, P, P, I64, P, F64P, F64P], ctypes.c_int),
        "pauli_autotune_commutator": ([P, P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       F64P, F64P], ctypes.c_int),
        "pauli_autotune_reset": ([], ctypes.c_int),
        "pauli_merge_geometry_fix": ([ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "pauli_batch_create": ([P, P, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(P)], ctypes.c_int),
        "pauli_batch_destroy": ([P], ctypes.c_int),
        "pauli_batch_rk4_step": ([P, P, P, ctypes.c_double, ctypes.c_int], ctypes.c_int),
        "pauli_batch_rk4_steps": ([P, P, P, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "pauli_batch_truncate": ([P, P], ctypes.c_int),
        "pauli_batch_counts": ([P, P, P], ctypes.c_int),
        "pauli_batch_norms": ([P, P, P], ctypes.c_int),
        "pauli_sum_set_precision": ([P, ctypes.c_int], ctypes.c_int),
        "pauli_sum_precision": ([P, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "pauli_mlp_param_count": ([], I64),
        "pauli_mlp_create": ([ctypes.c_int, ctypes.c_uint64, P, ctypes.POINTER(P)], ctypes.c_int),
        "pauli_mlp_destroy": ([P], ctypes.c_int),
        "pauli_mlp_get_params": ([P, P, I64], ctypes.c_int),
        "pauli_mlp_set_params": ([P, P, I64], ctypes.c_int),
        "pauli_mlp_features": ([P, P, P], ctypes.c_int),
        "pauli_mlp_logits": ([P, P, P], ctypes.c_int),
        "pauli_mlp_scores": ([P, P, ctypes.c_double, P], ctypes.c_int),
        "pauli_mlp_gradient": ([P, P, P, I64, I64, P, F64P], ctypes.c_int),
        "pauli_mlp_train_step": ([P, P, P, I64, I64, ctypes.c_float, F64P], ctypes.c_int),
        "pauli_mlp_labels": ([P, P, P], ctypes.c_int),
        "pauli_truncate_scored": ([P, ctypes.POINTER(pauli_trunc_policy), P, ctypes.c_double, P], ctypes.c_int),
        "pauli_rk4_step_mlp": ([P, P, ctypes.c_double, ctypes.POINTER(pauli_trunc_policy), P, P, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def declared_symbols() -> list[str]:
    """Names of the functions declared in include/paulistr.h."""
    import re
    hdr = os.path.join(_build.ROOT, "include", "paulistr.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"\b(pauli_[a-z_0-9]+)\s*\(", text)))


def _check(status: int, where: str):
    if status != PS_OK:
        raise PauliError(status, where)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def words_for(n_sites: int) -> int:
    """64-bit words per mask: 1 up to 64 sites, 2 up to 128, 4 up to 256."""
    return 1 if n_sites <= 64 else (2 if n_sites <= 128 else 4)


class PauliSum:
    """A device-resident Pauli sum (owns one ``pauli_sum*``).  Above 64 sites the masks v, w
    are (n, W) uint64 arrays (word k holds sites 64k+1 .. 64k+64), W = words_for(n_sites)."""

    def __init__(self, n_sites: int, capacity: int = 0, stream=None):
        lib = load()
        self._lib = lib
        self.n_sites = int(n_sites)
        self.W = words_for(self.n_sites)
        self.stream = _current_stream() if stream is None else ctypes.c_void_p(stream)
        h = ctypes.c_void_p()
        _check(lib.pauli_sum_create(self.n_sites, int(capacity), self.stream, ctypes.byref(h)), "pauli_sum_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and self._lib is not None:
            self._lib.pauli_sum_destroy(h)
            self.handle = None

    # ------------------------------------------------------------ data movement
    @classmethod
    def from_arrays(cls, n_sites: int, v, w, re, im, stream=None) -> "PauliSum":
        s = cls(n_sites, len(re), stream)
        s.upload(v, w, re, im)
        return s

    def upload(self, v, w, re, im):
        """Host upload (numpy arrays); order kept."""
        re, im = _f64(re), _f64(im)
        n = len(re)
        v = _u64(v).reshape(-1)
        w = _u64(w).reshape(-1)
        if len(v) != n * self.W or len(w) != n * self.W:
            raise ValueError(f"masks must hold {self.W} word(s) per string")
        U64P = ctypes.POINTER(ctypes.c_uint64)
        F64P = ctypes.POINTER(ctypes.c_double)
        _check(self._lib.pauli_sum_upload(self.handle, v.ctypes.data_as(U64P), w.ctypes.data_as(U64P),
                                          re.ctypes.data_as(F64P), im.ctypes.data_as(F64P), n), "pauli_sum_upload")

    def upload_device(self, v, w, re, im):
        """Device upload from torch CUDA tensors (uint64/int64 masks of W words per string, float64)."""
        n = int(re.numel())
        _check(self._lib.pauli_sum_upload_device(self.handle, ctypes.c_void_p(v.data_ptr()),
                                                 ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(re.data_ptr()),
                                                 ctypes.c_void_p(im.data_ptr()), n), "pauli_sum_upload_device")

    def __len__(self) -> int:
        n = ctypes.c_int64()
        _check(self._lib.pauli_sum_size(self.handle, ctypes.byref(n)), "pauli_sum_size")
        return int(n.value)

    def download(self):
        """(v, w, re, im) numpy arrays in canonical order (v, then w ascending)."""
        n = len(self)
        v = np.empty(n * self.W, np.uint64)
        w = np.empty(n * self.W, np.uint64)
        re = np.empty(n, np.float64)
        im = np.empty(n, np.float64)
        got = ctypes.c_int64()
        U64P = ctypes.POINTER(ctypes.c_uint64)
        F64P = ctypes.POINTER(ctypes.c_double)
        _check(self._lib.pauli_sum_download(self.handle, v.ctypes.data_as(U64P), w.ctypes.data_as(U64P),
                                            re.ctypes.data_as(F64P), im.ctypes.data_as(F64P), n,
                                            ctypes.byref(got)), "pauli_sum_download")
        if self.W > 1:
            return v.reshape(n, self.W), w.reshape(n, self.W), re, im
        return v, w, re, im

    def to_dict(self) -> dict:
        """{(v, w): c} with the masks as Python integers (any width)."""
        v, w, re, im = self.download()
        if self.W > 1:
            join = lambda row: sum(int(x) << (64 * k) for k, x in enumerate(row))  # noqa: E731
            return {(join(a), join(b)): complex(c, d) for a, b, c, d in zip(v, w, re, im)}
        return {(int(a), int(b)): complex(c, d) for a, b, c, d in zip(v, w, re, im)}

    def set_precision(self, coef_dtype: int) -> "PauliSum":
        """PS_COEF_F32 / PS_COEF_F32C: FP32 coefficients from now on (rounds the contents), the
        latter with FP32 arithmetic and compensated sums in merges; PS_COEF_F64: FP64."""
        _check(self._lib.pauli_sum_set_precision(self.handle, int(coef_dtype)), "pauli_sum_set_precision")
        return self

    def precision(self) -> int:
        d = ctypes.c_int()
        _check(self._lib.pauli_sum_precision(self.handle, ctypes.byref(d)), "pauli_sum_precision")
        return int(d.value)

    def sort_by_hash(self) -> "PauliSum":
        """Storage in the merge's output-hash order (for right operands; never for an H)."""
        _check(self._lib.pauli_sum_sort_by_hash(self.handle), "pauli_sum_sort_by_hash")
        return self

    def save(self, path: str, meta=()):
        """Checkpoint: the sum (canonical order), its precision and caller values (meta)."""
        m = np.ascontiguousarray(meta, dtype=np.float64)
        _check(self._lib.pauli_sum_save(self.handle, os.fsencode(path), m.ctypes.data_as(ctypes.c_void_p) if len(m) else None,
                                        len(m)), "pauli_sum_save")

    def load(self, path: str, meta_cap: int = 1 << 16) -> np.ndarray:
        """Resume from a checkpoint; returns the stored caller values."""
        m = np.zeros(meta_cap, np.float64)
        nm = ctypes.c_int64()
        _check(self._lib.pauli_sum_load(self.handle, os.fsencode(path), m.ctypes.data_as(ctypes.c_void_p), meta_cap,
                                        ctypes.byref(nm)), "pauli_sum_load")
        return m[:min(int(nm.value), meta_cap)].copy()

    def copy(self) -> "PauliSum":
        out = PauliSum(self.n_sites, len(self), self.stream.value)
        if self.precision() != PS_COEF_F64:
            out.set_precision(self.precision())
        _check(self._lib.pauli_sum_copy(self.handle, out.handle), "pauli_sum_copy")
        return out


def _h(s):
    return None if s is None else s.handle


def pauli_commutator(H: PauliSum, O: PauliSum, out: PauliSum | None = None) -> PauliSum:
    out = out if out is not None else PauliSum(O.n_sites, 0, O.stream.value)
    _check(load().pauli_commutator(H.handle, O.handle, out.handle), "pauli_commutator")
    return out


def pauli_multiply(A: PauliSum, B: PauliSum, out: PauliSum | None = None) -> PauliSum:
    """A B (operator product; A is the outer operand, at most 61439 strings)."""
    out = out if out is not None else PauliSum(B.n_sites, 0, B.stream.value)
    _check(load().pauli_multiply(A.handle, B.handle, out.handle), "pauli_multiply")
    return out


def pauli_add(A: PauliSum, alpha: complex, B: PauliSum, out: PauliSum | None = None) -> PauliSum:
    out = out if out is not None else PauliSum(A.n_sites, 0, A.stream.value)
    alpha = complex(alpha)
    _check(load().pauli_add(A.handle, alpha.real, alpha.imag, B.handle, out.handle), "pauli_add")
    return out


def pauli_truncate(O: PauliSum, pol: pauli_trunc_policy | None, keep: PauliSum | None = None, dt: float = 0.0):
    _check(load().pauli_truncate(O.handle, None if pol is None else ctypes.byref(pol), _h(keep), float(dt)),
           "pauli_truncate")
    return O


def pauli_rk4_step(H: PauliSum, O: PauliSum, dt: float, pol: pauli_trunc_policy | None = None,
                   keep: PauliSum | None = None):
    _check(load().pauli_rk4_step(H.handle, O.handle, float(dt), None if pol is None else ctypes.byref(pol),
                                 _h(keep)), "pauli_rk4_step")
    return O


def pauli_lanczos_step(H: PauliSum, O_prev: PauliSum, O_cur: PauliSum, b_prev: float,
                       pol: pauli_trunc_policy | None = None) -> float:
    """Returns b_n (0.0 when the Krylov space closed; then the sums are unchanged)."""
    b = ctypes.c_double()
    st = load().pauli_lanczos_step(H.handle, O_prev.handle, O_cur.handle, float(b_prev),
                                   None if pol is None else ctypes.byref(pol), ctypes.byref(b))
    if st == PS_ERR_KRYLOV_EXHAUSTED:
        return 0.0
    _check(st, "pauli_lanczos_step")
    return float(b.value)


# translation-symmetric generators (periodic chain of n_sites sites)
def pauli_ts_expand(G: PauliSum, out: PauliSum | None = None) -> PauliSum:
    out = out if out is not None else PauliSum(G.n_sites, 0, G.stream.value)
    _check(load().pauli_ts_expand(G.handle, out.handle), "pauli_ts_expand")
    return out


def pauli_ts_canonicalize(X: PauliSum, out: PauliSum | None = None) -> PauliSum:
    out = out if out is not None else PauliSum(X.n_sites, 0, X.stream.value)
    _check(load().pauli_ts_canonicalize(X.handle, out.handle), "pauli_ts_canonicalize")
    return out


def pauli_ts_commutator(H0: PauliSum, O0: PauliSum, out: PauliSum | None = None) -> PauliSum:
    out = out if out is not None else PauliSum(O0.n_sites, 0, O0.stream.value)
    _check(load().pauli_ts_commutator(H0.handle, O0.handle, out.handle), "pauli_ts_commutator")
    return out


def pauli_ts_norm(O0: PauliSum) -> float:
    r = ctypes.c_double()
    _check(load().pauli_ts_norm(O0.handle, ctypes.byref(r)), "pauli_ts_norm")
    return float(r.value)


def pauli_ts_lanczos_step(H0: PauliSum, O_prev: PauliSum, O_cur: PauliSum, b_prev: float,
                          pol: pauli_trunc_policy | None = None) -> float:
    b = ctypes.c_double()
    st = load().pauli_ts_lanczos_step(H0.handle, O_prev.handle, O_cur.handle, float(b_prev),
                                      None if pol is None else ctypes.byref(pol), ctypes.byref(b))
    if st == PS_ERR_KRYLOV_EXHAUSTED:
        return 0.0
    _check(st, "pauli_ts_lanczos_step")
    return float(b.value)


def pauli_trace_product(A: PauliSum, B: PauliSum) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(load().pauli_trace_product(A.handle, B.handle, ctypes.byref(re), ctypes.byref(im)), "pauli_trace_product")
    return complex(re.value, im.value)


def pauli_coefficients(O: PauliSum, v, w) -> np.ndarray:
    """Coefficients of the query strings (v[j], w[j]) in O (0 where absent): Tr(O P_q)/2^N,
    e.g. the two-point correlators Tr(O(t) Z_j)/2^N for all sites j."""
    v = np.ascontiguousarray(v, dtype=np.uint64)
    w = np.ascontiguousarray(w, dtype=np.uint64)
    n = len(v)
    re, im = np.zeros(n), np.zeros(n)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(load().pauli_coefficients(O.handle, ptr(v), ptr(w), n, ptr(re), ptr(im)), "pauli_coefficients")
    return re + 1j * im


def pauli_trace_product_noalloc(a_arrays, b_arrays, stream=None) -> complex:
    """Allocation-free Tr(AB)/2^N from device arrays: a_arrays/b_arrays are (v, w, re, im)
    torch CUDA tensors (64-bit masks, float64 coefficients)."""
    lib = load()
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(lib.pauli_trace_product_noalloc(*[ptr(t) for t in a_arrays], int(a_arrays[0].numel()),
                                           *[ptr(t) for t in b_arrays], int(b_arrays[0].numel()), st,
                                           ctypes.byref(re), ctypes.byref(im)), "pauli_trace_product_noalloc")
    return complex(re.value, im.value)


def pauli_norm(O: PauliSum) -> float:
    r = ctypes.c_double()
    _check(load().pauli_norm(O.handle, ctypes.byref(r)), "pauli_norm")
    return float(r.value)


def pauli_last_merge_stats() -> dict:
    st = pauli_merge_stats()
    _check(load().pauli_last_merge_stats(ctypes.byref(st)), "pauli_last_merge_stats")
    return {k: int(getattr(st, k)) for k, _ in pauli_merge_stats._fields_}


def pauli_profile_enable(on: bool = True):
    _check(load().pauli_profile_enable(1 if on else 0), "pauli_profile_enable")


def pauli_profile_report() -> dict:
    """{kernel: (launches, total_ms)} since profiling was enabled."""
    import json
    lib = load()
    need = ctypes.c_int64()
    lib.pauli_profile_report(None, 0, ctypes.byref(need))
    buf = ctypes.create_string_buffer(int(need.value) + 64)
    _check(lib.pauli_profile_report(buf, len(buf), ctypes.byref(need)), "pauli_profile_report")
    return {k: (int(v[0]), float(v[1])) for k, v in json.loads(buf.value.decode()).items()}


def pauli_launch_count() -> int:
    return int(load().pauli_launch_count())


def pauli_debug_divide(x, b: float, stream=None):
    """In-place division of a float64 CUDA tensor by b with the library's Lanczos division."""
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _check(load().pauli_debug_divide(ctypes.c_void_p(x.data_ptr()), int(x.numel()), float(b), st),
           "pauli_debug_divide")
    return x


def pauli_debug_fail_alloc_after(n: int):
    _check(load().pauli_debug_fail_alloc_after(int(n)), "pauli_debug_fail_alloc_after")


def pauli_debug_mlp_wait(no_products: int = 0, wait_limit: int = 1 << 26):
    _check(load().pauli_debug_mlp_wait(int(no_products), int(wait_limit)), "pauli_debug_mlp_wait")


def pauli_debug_general_truncation(on: int = 1):
    _check(load().pauli_debug_general_truncation(int(on)), "pauli_debug_general_truncation")


def pauli_debug_output_hash(v, w) -> np.ndarray:
    """The merge's 32-bit output hash of host strings (host-side; for tests)."""
    v, w = _u64(v), _u64(w)
    out = np.zeros(len(v), np.uint32)
    _check(load().pauli_debug_output_hash(v.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                                          len(v), out.ctypes.data_as(ctypes.c_void_p)), "pauli_debug_output_hash")
    return out


# ------------------------------------------------------------------ learned truncation
def _dev(t):
    return ctypes.c_void_p(t.data_ptr())


class PauliMLP:
    """The learned truncation scorer (owns one ``pauli_mlp*``); see include/paulistr.h."""

    def __init__(self, n_sites: int, seed: int = 0, stream=None):
        lib = load()
        self._lib = lib
        self.n_sites = int(n_sites)
        self.stream = _current_stream() if stream is None else ctypes.c_void_p(stream)
        h = ctypes.c_void_p()
        _check(lib.pauli_mlp_create(self.n_sites, ctypes.c_uint64(int(seed)), self.stream, ctypes.byref(h)),
               "pauli_mlp_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and self._lib is not None:
            self._lib.pauli_mlp_destroy(h)
            self.handle = None


def pauli_mlp_param_count() -> int:
    return int(load().pauli_mlp_param_count())


def pauli_mlp_get_params(m: PauliMLP) -> np.ndarray:
    n = pauli_mlp_param_count()
    out = np.empty(n, np.float32)
    _check(load().pauli_mlp_get_params(m.handle, out.ctypes.data_as(ctypes.c_void_p), n), "pauli_mlp_get_params")
    return out


def pauli_mlp_set_params(m: PauliMLP, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().pauli_mlp_set_params(m.handle, p.ctypes.data_as(ctypes.c_void_p), len(p)), "pauli_mlp_set_params")


def pauli_mlp_features(m: PauliMLP, O: PauliSum):
    """BF16 bit patterns of the 80 features of O's strings (storage order): int16 CUDA tensor [n, 80]."""
    import torch
    x = torch.empty((len(O), 80), dtype=torch.int16, device="cuda")
    _check(load().pauli_mlp_features(m.handle, O.handle, _dev(x)), "pauli_mlp_features")
    return x


def pauli_mlp_logits(m: PauliMLP, O: PauliSum):
    import torch
    z = torch.empty(len(O), dtype=torch.float32, device="cuda")
    _check(load().pauli_mlp_logits(m.handle, O.handle, _dev(z)), "pauli_mlp_logits")
    return z


def pauli_mlp_scores(m: PauliMLP, O: PauliSum, gamma_dt: float = 0.0):
    import torch
    sc = torch.empty(len(O), dtype=torch.float64, device="cuda")
    _check(load().pauli_mlp_scores(m.handle, O.handle, float(gamma_dt), _dev(sc)), "pauli_mlp_scores")
    return sc


def pauli_mlp_gradient(m: PauliMLP, X: PauliSum, labels, i0: int = 0, nb: int | None = None):
    """(gradient as a float32 numpy array, loss) over records [i0, i0 + nb) of X."""
    nb = len(X) - i0 if nb is None else nb
    g = np.empty(pauli_mlp_param_count(), np.float32)
    loss = ctypes.c_double()
    _check(load().pauli_mlp_gradient(m.handle, X.handle, _dev(labels), int(i0), int(nb),
                                     g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss)), "pauli_mlp_gradient")
    return g, float(loss.value)


def pauli_mlp_train_step(m: PauliMLP, X: PauliSum, labels, i0: int, nb: int, lr: float, want_loss: bool = False):
    loss = ctypes.c_double()
    _check(load().pauli_mlp_train_step(m.handle, X.handle, _dev(labels), int(i0), int(nb), float(lr),
                                       ctypes.byref(loss) if want_loss else None), "pauli_mlp_train_step")
    return float(loss.value) if want_loss else None


def pauli_mlp_labels(X: PauliSum, target: PauliSum):
    """float32 CUDA tensor: 1 where X's string (storage order) is present in target."""
    import torch
    y = torch.empty(len(X), dtype=torch.float32, device="cuda")
    _check(load().pauli_mlp_labels(X.handle, target.handle, _dev(y)), "pauli_mlp_labels")
    return y


def pauli_truncate_scored(O: PauliSum, pol: pauli_trunc_policy | None, score, keep: PauliSum | None = None,
                          dt: float = 0.0):
    """Truncation with the top-k ranked by score (float64 CUDA tensor, O's storage order)."""
    _check(load().pauli_truncate_scored(O.handle, None if pol is None else ctypes.byref(pol), _h(keep), float(dt),
                                        _dev(score)), "pauli_truncate_scored")
    return O


def pauli_rk4_step_mlp(H: PauliSum, O: PauliSum, dt: float, pol: pauli_trunc_policy | None = None,
                       keep: PauliSum | None = None, model: PauliMLP | None = None,
                       cand_out: PauliSum | None = None):
    _check(load().pauli_rk4_step_mlp(H.handle, O.handle, float(dt), None if pol is None else ctypes.byref(pol),
                                     _h(keep), None if model is None else model.handle, _h(cand_out)),
           "pauli_rk4_step_mlp")
    return O


def pauli_sum_set_precision(S: PauliSum, coef_dtype: int) -> PauliSum:
    return S.set_precision(coef_dtype)


def pauli_sum_precision(S: PauliSum) -> int:
    return S.precision()


# ------------------------------------------------------------------ batched instances
class PauliBatch:
    """Per-instance H coefficients and caps of instance-tagged sums (owns one ``pauli_batch*``)."""

    def __init__(self, H: PauliSum, hcoef, tag_shift: int, caps=None):
        lib = load()
        self._lib = lib
        hc = np.ascontiguousarray(hcoef, dtype=np.float64)
        if hc.ndim != 2:
            raise ValueError("hcoef must be [n_inst, |H|]")
        self.n_inst = int(hc.shape[0])
        self.tag_shift = int(tag_shift)
        cp = None if caps is None else np.ascontiguousarray(caps, dtype=np.int64)
        h = ctypes.c_void_p()
        _check(lib.pauli_batch_create(H.handle, hc.ctypes.data_as(ctypes.c_void_p), self.n_inst, self.tag_shift,
                                      None if cp is None else cp.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)),
               "pauli_batch_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and self._lib is not None:
            self._lib.pauli_batch_destroy(h)
            self.handle = None


def pauli_batch_rk4_step(B: PauliBatch, H: PauliSum, O: PauliSum, dt: float, trim_stages: int = 0) -> PauliSum:
    _check(load().pauli_batch_rk4_step(B.handle, H.handle, O.handle, float(dt), int(trim_stages)),
           "pauli_batch_rk4_step")
    return O


def pauli_batch_rk4_steps(B: PauliBatch, H: PauliSum, O: PauliSum, dt: float, n_steps: int,
                          trim_stages: int = 0) -> PauliSum:
    done = ctypes.c_int()
    _check(load().pauli_batch_rk4_steps(B.handle, H.handle, O.handle, float(dt), int(trim_stages), int(n_steps),
                                        ctypes.byref(done)), "pauli_batch_rk4_steps")
    return O


def pauli_batch_truncate(B: PauliBatch, O: PauliSum) -> PauliSum:
    _check(load().pauli_batch_truncate(B.handle, O.handle), "pauli_batch_truncate")
    return O


def pauli_batch_counts(B: PauliBatch, O: PauliSum) -> np.ndarray:
    out = np.zeros(B.n_inst, np.int64)
    _check(load().pauli_batch_counts(B.handle, O.handle, out.ctypes.data_as(ctypes.c_void_p)), "pauli_batch_counts")
    return out


def pauli_batch_norms(B: PauliBatch, O: PauliSum) -> np.ndarray:
    out = np.zeros(B.n_inst, np.float64)
    _check(load().pauli_batch_norms(B.handle, O.handle, out.ctypes.data_as(ctypes.c_void_p)), "pauli_batch_norms")
    return out


# ------------------------------------------------------------------ autotuner
def pauli_autotune_commutator(H: PauliSum, O: PauliSum, reps: int = 3) -> dict:
    """Time [H, O] over the merge geometries and keep the fastest for its size class."""
    bt, q = ctypes.c_int(), ctypes.c_int()
    best, default = ctypes.c_double(), ctypes.c_double()
    _check(load().pauli_autotune_commutator(H.handle, O.handle, int(reps), ctypes.byref(bt), ctypes.byref(q),
                                            ctypes.byref(best), ctypes.byref(default)), "pauli_autotune_commutator")
    return {"bin_target": int(bt.value), "quota": int(q.value), "best_ms": float(best.value),
            "default_ms": float(default.value)}


def pauli_autotune_reset():
    _check(load().pauli_autotune_reset(), "pauli_autotune_reset")


def pauli_merge_geometry_fix(bin_target: int, quota: int):
    _check(load().pauli_merge_geometry_fix(int(bin_target), int(quota)), "pauli_merge_geometry_fix")


# ------------------------------------------------------------------ the remaining C names
# Module-level functions with the C ABI's names for the calls the classes above wrap
# (construction, destruction, data movement, status strings); argument marshalling only.
def pauli_status_string(status: int) -> str:
    return load().pauli_status_string(int(status)).decode()


def pauli_last_cuda_error() -> str:
    return load().pauli_last_cuda_error().decode()


def pauli_sum_create(n_sites: int, capacity: int = 0, stream=None) -> PauliSum:
    return PauliSum(n_sites, capacity, stream)


def pauli_sum_destroy(S: PauliSum):
    S.__del__()


def pauli_sum_upload(S: PauliSum, v, w, re, im) -> PauliSum:
    S.upload(v, w, re, im)
    return S


def pauli_sum_upload_device(S: PauliSum, v, w, re, im) -> PauliSum:
    S.upload_device(v, w, re, im)
    return S


def pauli_sum_size(S: PauliSum) -> int:
    return len(S)


def pauli_sum_n_sites(S: PauliSum) -> int:
    n = ctypes.c_int()
    _check(load().pauli_sum_n_sites(S.handle, ctypes.byref(n)), "pauli_sum_n_sites")
    return int(n.value)


def pauli_sum_download(S: PauliSum):
    """(v, w, re, im) numpy arrays in canonical order."""
    return S.download()


def pauli_sum_download_device(S: PauliSum, out=None):
    """(v, w, re, im) in storage order: int64 bit patterns of the masks and float64, as new CUDA
    tensors, or written into `out` (four tensors of at least the sum's size: CUDA tensors or
    pinned host tensors, which the library writes over the host link; complete once the sum's
    stream has run the call).  Returns the four tensors cut to the sum's size."""
    import torch
    m = len(S)
    if out is None:
        t = [torch.empty(m * S.W, dtype=torch.int64, device="cuda"), torch.empty(m * S.W, dtype=torch.int64, device="cuda"),
             torch.empty(m, dtype=torch.float64, device="cuda"), torch.empty(m, dtype=torch.float64, device="cuda")]
        cap = m
    else:
        t = list(out)
        cap = min(int(t[2].numel()), int(t[3].numel()), int(t[0].numel()) // S.W, int(t[1].numel()) // S.W)
    got = ctypes.c_int64()
    _check(load().pauli_sum_download_device(S.handle, *[ctypes.c_void_p(x.data_ptr()) for x in t], cap,
                                            ctypes.byref(got)), "pauli_sum_download_device")
    if out is not None:
        t = [t[0][:m * S.W], t[1][:m * S.W], t[2][:m], t[3][:m]]
    if S.W > 1:
        t[0], t[1] = t[0].view(m, S.W), t[1].view(m, S.W)
    return tuple(t)


def pauli_sum_copy(src: PauliSum, dst: PauliSum | None = None) -> PauliSum:
    if dst is None:
        return src.copy()
    _check(load().pauli_sum_copy(src.handle, dst.handle), "pauli_sum_copy")
    return dst


def pauli_sum_sort_by_hash(S: PauliSum) -> PauliSum:
    return S.sort_by_hash()


def pauli_sum_save(S: PauliSum, path: str, meta=()):
    S.save(path, meta)


def pauli_sum_load(S: PauliSum, path: str, meta_cap: int = 1 << 16) -> np.ndarray:
    return S.load(path, meta_cap)


def pauli_mlp_create(n_sites: int, seed: int = 0, stream=None) -> PauliMLP:
    return PauliMLP(n_sites, seed, stream)


def pauli_mlp_destroy(m: PauliMLP):
    m.__del__()


def pauli_batch_create(H: PauliSum, hcoef, tag_shift: int, caps=None) -> PauliBatch:
    return PauliBatch(H, hcoef, tag_shift, caps)


def pauli_batch_destroy(B: PauliBatch):
    B.__del__()
