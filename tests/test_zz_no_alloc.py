"""The allocation-free trace product, for callers that cannot allocate device memory
(code under another framework's allocator or memory budget, plug-ins handed only
pre-allocated buffers).  It must give the same exactly rounded Tr(AB)/2^N as the
oracle and as pauli_trace_product, call after call, although every call reuses one
fixed scratch array inside the library.

This file is collected last on purpose: it runs after every other test, and it also
passes on its own in a fresh process."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
from paper_2410_09654_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2410_09654_gb300 import paulistr as ps  # noqa: E402

REL_TOL = 1e-12  # the FP64 tolerance of the parity tests
ONES = np.uint64(0xFFFFFFFFFFFFFFFF)  # Y on all 64 sites: the key the scratch table keeps apart


def _operands(seed, n_sites, na, nb, shared):
    rng = np.random.default_rng(seed)
    v, w = I.random_strings(rng, n_sites, na + nb - shared)
    a = (v[:na], w[:na], rng.standard_normal(na), rng.standard_normal(na) * (seed % 2))
    b = (v[na - shared:], w[na - shared:], rng.standard_normal(nb) * 1e-3, rng.standard_normal(nb))
    return a, b


def _with_ones(arrays, coef):
    """The operand with its first string replaced by the all-ones key (v = w = ~0)."""
    v, w, re, im = (np.array(x, copy=True) for x in arrays)
    keep = ~((v == ONES) & (w == ONES))
    v, w, re, im = v[keep], w[keep], re[keep], im[keep]
    v[0], w[0], re[0], im[0] = ONES, ONES, coef.real, coef.imag
    return v, w, re, im


def _device(arrays):
    v, w, re, im = arrays
    as_i64 = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint64).view(np.int64)).cuda()
    return (as_i64(v), as_i64(w), torch.from_numpy(np.ascontiguousarray(re)).cuda(),
            torch.from_numpy(np.ascontiguousarray(im)).cuda())


def _close(x: complex, y: complex):
    for p, q in ((x.real, y.real), (x.imag, y.imag)):
        assert abs(p - q) <= REL_TOL * abs(q), (x, y)


def _check(a, b):
    """noalloc result == oracle == pauli_trace_product (all exactly rounded), with the
    library's allocation hook armed so that any device allocation inside the call fails."""
    want = orc.trace_product(orc.Op(64, *a), orc.Op(64, *b))
    lib_val = ps.pauli_trace_product(ps.PauliSum.from_arrays(64, *a), ps.PauliSum.from_arrays(64, *b))
    da, db = _device(a), _device(b)
    torch.cuda.synchronize()
    ps.pauli_debug_fail_alloc_after(1)  # the next library allocation would return PS_ERR_NOMEM
    try:
        got = ps.pauli_trace_product_noalloc(da, db)
    finally:
        ps.pauli_debug_fail_alloc_after(0)
    torch.cuda.synchronize()
    _close(got, want)
    assert got == want == lib_val  # the exactly rounded sums


def test_noalloc_matches_oracle_on_two_calls_in_row():
    ps.load(build_if_missing=True)
    cases = [_operands(11, 64, 120000, 90000, 40000),   # first call fills most of the table
             _operands(12, 40, 3000, 20000, 1500)]      # second call: smaller table, stale scratch around it
    for a, b in cases:
        _check(a, b)


def test_noalloc_all_ones_key_then_without_it():
    """The all-ones key is stored apart from the table; a stale index from the previous
    call must not leak into the next one."""
    ps.load(build_if_missing=True)
    a, b = _operands(21, 64, 5000, 7000, 2000)
    _check(_with_ones(a, 0.75 - 0.5j), _with_ones(b, -1.25 + 2.0j))  # both hold Y...Y
    a2, b2 = _operands(22, 64, 5000, 7000, 2000)
    _check(a2, _with_ones(b2, 3.0 + 0.0j))  # only the larger operand holds it: no match


def test_noalloc_largest_accepted_operand():
    """The smaller operand at exactly the scratch limit (131072 strings: every table slot
    pair in use at load 0.5)."""
    ps.load(build_if_missing=True)
    a, b = _operands(23, 64, 131072, 140000, 60000)
    _check(a, b)


def test_noalloc_rejects_operands_beyond_its_scratch():
    ps.load(build_if_missing=True)
    a, b = _operands(13, 64, 131073, 131073, 10)
    with pytest.raises(ps.PauliError) as e:
        ps.pauli_trace_product_noalloc(_device(a), _device(b))
    assert e.value.status == ps.PS_ERR_CAPACITY
