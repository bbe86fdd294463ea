"""The C-ABI library builds, loads and exports every symbol that include/paulistr.h
declares (no compute calls: runs without a GPU)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

from paper_2410_09654_gb300 import build as B
from paper_2410_09654_gb300 import paulistr as ps

HDR = os.path.join(B.ROOT, "include", "paulistr.h")


@pytest.fixture(scope="module")
def lib():
    try:
        B.build()
    except RuntimeError as e:  # no nvcc here
        pytest.skip(str(e))
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_path():
    names = ps.declared_symbols()
    for need in ("pauli_sum_create", "pauli_commutator", "pauli_truncate", "pauli_rk4_step",
                 "pauli_lanczos_step", "pauli_trace_product"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pauli_\w+)", out))
    missing = [s for s in ps.declared_symbols() if s not in exported]
    assert not missing, missing
    for s in ps.declared_symbols():
        getattr(lib, s)  # resolvable through dlsym


def test_binding_signatures_cover_header(lib):
    l = ps.load()
    for s in ps.declared_symbols():
        assert getattr(l, s).argtypes is not None, s


def test_status_strings_without_gpu(lib):
    l = ps.load()
    assert l.pauli_status_string(0) == b"ok"
    assert b"Krylov" in l.pauli_status_string(ps.PS_ERR_KRYLOV_EXHAUSTED)


def test_invalid_arguments_are_rejected_on_the_host(lib):
    l = ps.load()
    h = ctypes.c_void_p()
    assert l.pauli_sum_create(0, 0, None, ctypes.byref(h)) == ps.PS_ERR_INVALID
    assert l.pauli_sum_create(257, 0, None, ctypes.byref(h)) == ps.PS_ERR_INVALID  # masks of at most 4 words
    assert l.pauli_commutator(None, None, None) == ps.PS_ERR_INVALID
    assert l.pauli_lanczos_step(None, None, None, 0.0, None, None) == ps.PS_ERR_INVALID


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(B.ROOT, "paper_2410_09654_gb300")
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_every_declared_function_has_a_binding_of_the_same_name():
    from paper_2410_09654_gb300 import paulistr as ps
    missing = [n for n in ps.declared_symbols() if not callable(getattr(ps, n, None))]
    assert not missing, missing


def test_output_hash_hook_is_linear_without_gpu(lib):
    """The merge's output hash is GF(2)-linear: F(a ^ b) = F(a) ^ F(b) (host-side hook)."""
    import numpy as np
    rng = np.random.default_rng(3)
    a = rng.integers(0, 2**63, size=(2, 200), dtype=np.int64).astype(np.uint64) * np.uint64(2)
    b = rng.integers(0, 2**63, size=(2, 200), dtype=np.int64).astype(np.uint64) + np.uint64(1)
    fa = ps.pauli_debug_output_hash(a[0], a[1])
    fb = ps.pauli_debug_output_hash(b[0], b[1])
    fab = ps.pauli_debug_output_hash(a[0] ^ b[0], a[1] ^ b[1])
    assert np.array_equal(fab, fa ^ fb)
    assert not ps.pauli_debug_output_hash(np.zeros(1, np.uint64), np.zeros(1, np.uint64)).any()
    assert len(set(fa.tolist())) > 190  # spreads distinct keys
