"""The module-level bindings with the C names (marshalling only) on a small sum."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2410_09654_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2410_09654_gb300 import paulistr as ps  # noqa: E402


def test_module_level_bindings(tmp_path):
    ps.load(build_if_missing=True)
    n = 20
    arr = I.random_sum(1, n, 500, kind="complex")
    S = ps.pauli_sum_create(n, 0)
    ps.pauli_sum_upload(S, *arr)
    assert ps.pauli_sum_size(S) == len(arr[0]) and ps.pauli_sum_n_sites(S) == n
    v, w, re, im = ps.pauli_sum_download_device(S)
    D = ps.pauli_sum_create(n)
    ps.pauli_sum_upload_device(D, v, w, re, im)
    C = ps.pauli_sum_copy(D)
    ps.pauli_sum_sort_by_hash(C)
    a, b = ps.pauli_sum_download(S), ps.pauli_sum_download(C)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    ps.pauli_sum_save(C, str(tmp_path / "c.ckp"), [1.5])
    E = ps.pauli_sum_create(n)
    assert list(ps.pauli_sum_load(E, str(tmp_path / "c.ckp"))) == [1.5]
    assert ps.pauli_status_string(ps.PS_ERR_IO) == "checkpoint file error"
    assert isinstance(ps.pauli_last_cuda_error(), str)
    m = ps.pauli_mlp_create(n, 3)
    ps.pauli_mlp_destroy(m)
    H = ps.PauliSum.from_arrays(n + 2, *I.random_field_xxz_chain(n, 1.0, 0).arrays()[:2],
                                np.ones(3 * (n - 1) + n), np.zeros(3 * (n - 1) + n))
    B = ps.pauli_batch_create(H, np.ones((3, len(H))), n)
    ps.pauli_batch_destroy(B)
    for x in (S, D, C, E, H):
        ps.pauli_sum_destroy(x)


def _pinned(a):
    """A copy of numpy array a in pinned host memory (mapped into the device's address space)."""
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def test_upload_rejects_a_repeated_string_and_keeps_distinct_ones():
    n = 64
    v, w, re, im = I.random_sum(3, n, 20000, kind="real")
    ones = np.uint64(0xFFFFFFFFFFFFFFFF)  # Y on every site
    v2, w2 = np.append(v, ones), np.append(w, ones)
    re2, im2 = np.append(re, 1.0), np.append(im, 0.0)
    S = ps.PauliSum.from_arrays(n, v2, w2, re2, im2)  # all distinct, the all-ones key once
    assert len(S) == len(re2)
    for dup in (17, len(re2) - 1):  # a random string, then the all-ones key, repeated
        with pytest.raises(ps.PauliError):
            ps.PauliSum.from_arrays(n, np.append(v2, v2[dup]), np.append(w2, w2[dup]),
                                    np.append(re2, 2.0), np.append(im2, 0.0))
    with pytest.raises(ps.PauliError):  # the same through pinned host arrays
        ps.PauliSum.from_arrays(n, *[_pinned(np.append(x, x[5])) for x in (v2, w2, re2, im2)])


def test_upload_from_pinned_host_arrays_equals_pageable():
    n = 64
    arr = I.random_sum(4, n, 300000, kind="complex")
    A = ps.PauliSum.from_arrays(n, *arr)
    B = ps.PauliSum.from_arrays(n, *[_pinned(x) for x in arr])
    a, b = A.download(), B.download()
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    # storage order is the given order on both paths
    da, db = ps.pauli_sum_download_device(A), ps.pauli_sum_download_device(B)
    assert all(torch.equal(x, y) for x, y in zip(da, db))


def test_download_device_into_pinned_host_memory_and_refusals():
    import ctypes
    n = 64
    arr = I.random_sum(5, n, 100000, kind="complex")
    S = ps.PauliSum.from_arrays(n, *arr)
    m = len(S)
    host = [torch.empty(m, dtype=dt).pin_memory() for dt in (torch.int64, torch.int64, torch.float64, torch.float64)]
    got = ctypes.c_int64()
    ps._check(ps.load().pauli_sum_download_device(S.handle, *[ctypes.c_void_p(t.data_ptr()) for t in host], m,
                                                   ctypes.byref(got)), "download_device")
    torch.cuda.synchronize()
    dev = ps.pauli_sum_download_device(S)  # the same storage order
    assert got.value == m
    for h, d in zip(host, dev):
        assert torch.equal(h, d.cpu().view(h.dtype))
    # pageable host memory is refused, nothing written
    page = [np.full(m, 7, np.int64), np.full(m, 7, np.int64), np.full(m, 7.0), np.full(m, 7.0)]
    rc = ps.load().pauli_sum_download_device(S.handle, *[ctypes.c_void_p(x.ctypes.data) for x in page], m,
                                             ctypes.byref(got))
    assert rc == ps.PS_ERR_INVALID and all((x == 7).all() for x in page)
    # and the device upload refuses pageable arrays too
    rc = ps.load().pauli_sum_upload_device(S.handle, *[ctypes.c_void_p(x.ctypes.data) for x in page], m)
    assert rc == ps.PS_ERR_INVALID
    assert len(S) == m
