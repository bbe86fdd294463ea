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
