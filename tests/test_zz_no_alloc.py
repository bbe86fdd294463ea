"""The allocation-free trace product, for callers that cannot allocate device memory
(code under another framework's allocator or memory budget, plug-ins handed only
pre-allocated buffers).  It must give the same exactly rounded Tr(AB)/2^N as
pauli_trace_product, call after call, although every call reuses one fixed scratch
array inside the library.

This file is collected last on purpose: it runs after every other test, and it also
passes on its own in a fresh process."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2410_09654_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2410_09654_gb300 import paulistr as ps  # noqa: E402

REL_TOL = 1e-12  # the FP64 tolerance of the parity tests


def _operands(seed, n_sites, na, nb, shared):
    rng = np.random.default_rng(seed)
    v, w = I.random_strings(rng, n_sites, na + nb - shared)
    a = (v[:na], w[:na], rng.standard_normal(na), rng.standard_normal(na) * (seed % 2))
    b = (v[na - shared:], w[na - shared:], rng.standard_normal(nb) * 1e-3, rng.standard_normal(nb))
    return a, b


def _device(arrays):
    v, w, re, im = arrays
    as_i64 = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint64).view(np.int64)).cuda()
    return (as_i64(v), as_i64(w), torch.from_numpy(np.ascontiguousarray(re)).cuda(),
            torch.from_numpy(np.ascontiguousarray(im)).cuda())


def _close(x: complex, y: complex):
    for p, q in ((x.real, y.real), (x.imag, y.imag)):
        assert abs(p - q) <= REL_TOL * abs(q), (x, y)


def test_noalloc_matches_trace_product_on_two_calls_in_row():
    ps.load(build_if_missing=True)
    cases = [_operands(11, 64, 120000, 90000, 40000),   # first call fills most of the table
             _operands(12, 40, 3000, 20000, 1500)]      # second call: smaller table, stale scratch around it
    for a, b in cases:
        want = ps.pauli_trace_product(ps.PauliSum.from_arrays(64, *a), ps.PauliSum.from_arrays(64, *b))
        got = ps.pauli_trace_product_noalloc(_device(a), _device(b))
        torch.cuda.synchronize()
        _close(got, want)
        assert got == want  # both are the exactly rounded sums


def test_noalloc_rejects_operands_beyond_its_scratch():
    ps.load(build_if_missing=True)
    a, b = _operands(13, 64, 131073, 131073, 10)
    with pytest.raises(ps.PauliError) as e:
        ps.pauli_trace_product_noalloc(_device(a), _device(b))
    assert e.value.status == ps.PS_ERR_CAPACITY
