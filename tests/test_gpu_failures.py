"""Failure paths, all made on the host: device allocations that fail (the library's
allocation hook), a merge whose strings cannot be separated by its hash (inputs built in the
kernel of the output hash), non-finite coefficients, and small download capacities.  Each
call must return its status, leave its operands as they were, trap nothing, and leave the
library usable: the next call agrees with the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
from paper_2410_09654_gb300 import inputs as I

from gpu_util import assert_match

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2410_09654_gb300 import paulistr as ps  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ps.load(build_if_missing=True)
    yield
    ps.pauli_debug_fail_alloc_after(0)


def _arrays(S):
    return tuple(np.array(x, copy=True) for x in S.download())


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def _each_failing_allocation(run, operands, limit=200):
    """Make the 1st, 2nd, ... allocation of run() fail until one run needs no more; every
    failed run returns PS_ERR_NOMEM and leaves the operands unchanged."""
    before = [_arrays(S) for S in operands]
    failures = 0
    for n in range(1, limit):
        ps.pauli_debug_fail_alloc_after(n)
        try:
            run()
        except ps.PauliError as e:
            assert e.status == ps.PS_ERR_NOMEM, e
            failures += 1
            torch.cuda.synchronize()
            for S, b in zip(operands, before):
                assert _same(_arrays(S), b), f"operand changed by a failed call (allocation {n})"
            continue
        finally:
            ps.pauli_debug_fail_alloc_after(0)
        return failures
    raise AssertionError("the call kept allocating")


def test_allocation_failures_in_commutator_rk4_and_lanczos():
    n = 10
    hb = I.tilted_ising_chain(n)
    H = ps.PauliSum.from_arrays(n, *hb.arrays())
    Hr = orc.Op(n, *hb.arrays())
    rng = np.random.default_rng(5)
    v, w = I.random_strings(rng, n, 400, max_support=5)
    Oa = (v, w, rng.standard_normal(400), np.zeros(400))
    O = ps.PauliSum.from_arrays(n, *Oa)
    Or = orc.Op(n, *Oa)

    out = ps.PauliSum(n)
    assert _each_failing_allocation(lambda: ps.pauli_commutator(H, O, out), [H, O]) > 0
    assert_match(out.download(), orc.commutator(Hr, Or), what="commutator after failures")

    pol = ps.policy(max_weight=6, cutoff=1e-10)
    assert _each_failing_allocation(lambda: ps.pauli_rk4_step(H, O, 0.05, pol), [H]) > 0
    # the failed steps left O as it was: the one that succeeded is the first step from Oa
    assert_match(O.download(), orc.rk4_step(Hr, Or, 0.05, max_weight=6, cutoff=1e-10), what="rk4 after failures")

    prev, cur = ps.PauliSum(n), ps.PauliSum.from_arrays(n, *I.single(n, "X", 1).arrays())
    state = {"b": 0.0}

    def lanczos():
        state["b"] = ps.pauli_lanczos_step(H, prev, cur, 0.0, ps.policy(cutoff=1e-10))

    assert _each_failing_allocation(lanczos, [prev, cur]) > 0
    rb, rn = orc.lanczos_step(Hr, orc.Op.empty(n), orc.Op(n, *I.single(n, "X", 1).arrays()), 0.0, cutoff=1e-10)
    assert state["b"] == rb
    assert_match(cur.download(), rn, what="lanczos after failures")


def _hash_kernel_keys(count):
    """`count` distinct 64-site strings whose whole 32-bit output hash is zero: a merge bins
    them together and no further hash bit separates them."""
    cols = []
    for i in range(128):
        v = np.array([1 << i if i < 64 else 0], np.uint64)
        w = np.array([1 << (i - 64) if i >= 64 else 0], np.uint64)
        cols.append(int(ps.pauli_debug_output_hash(v, w)[0]))
    # null space of the 32 x 128 GF(2) matrix whose column i is cols[i]
    rows = [(cols[i], 1 << i) for i in range(128)]  # (image, combination of unit vectors)
    basis, null = {}, []
    for img, comb in rows:
        while img:
            top = img.bit_length() - 1
            if top not in basis:
                basis[top] = (img, comb)
                break
            img ^= basis[top][0]
            comb ^= basis[top][1]
        if img == 0:
            null.append(comb)
    k = (count - 1).bit_length()
    assert len(null) >= k
    keys = []
    for m in range(1, count + 1):
        comb = 0
        for j in range(k + 1):
            if (m >> j) & 1:
                comb ^= null[j]
        keys.append(comb)
    v = np.array([c & ((1 << 64) - 1) for c in keys], np.uint64)
    w = np.array([c >> 64 for c in keys], np.uint64)
    assert not ps.pauli_debug_output_hash(v, w).any()
    assert len(set(zip(v.tolist(), w.tolist()))) == count
    return v, w


def test_merge_that_cannot_split_returns_table_full():
    n = 64
    v, w = _hash_kernel_keys(4096)
    rng = np.random.default_rng(9)
    A = ps.PauliSum.from_arrays(n, v, w, rng.standard_normal(len(v)), np.zeros(len(v)))
    before = _arrays(A)
    B = ps.PauliSum(n)
    out = ps.PauliSum(n)
    with pytest.raises(ps.PauliError) as e:
        ps.pauli_add(A, 1.0, B, out)
    assert e.value.status == ps.PS_ERR_TABLE_FULL
    assert _same(_arrays(A), before)
    # the library is still usable, and a merge of fewer colliding strings works
    m = 500  # 1000 entries and 500 distinct strings: one merge pass holds them
    C = ps.PauliSum.from_arrays(n, v[:m], w[:m], np.ones(m), np.zeros(m))
    ps.pauli_add(C, 0.5, C.copy(), out)
    Cr = orc.Op(n, v[:m], w[:m], np.ones(m), np.zeros(m))
    assert_match(out.download(), orc.axpy(Cr, 0.5, Cr), what="merge of 500 colliding strings")


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_uploads_reject_non_finite_coefficients(bad):
    n = 8
    v, w = np.array([1, 2, 3], np.uint64), np.array([0, 1, 0], np.uint64)
    for re, im in (([1.0, bad, 2.0], [0.0, 0.0, 0.0]), ([1.0, 0.5, 2.0], [0.0, 0.0, bad])):
        S = ps.PauliSum(n)
        with pytest.raises(ps.PauliError) as e:
            S.upload(v, w, np.array(re), np.array(im))
        assert e.value.status == ps.PS_ERR_INVALID
        assert len(S) == 0
        dv = torch.from_numpy(v.view(np.int64)).cuda()
        dw = torch.from_numpy(w.view(np.int64)).cuda()
        with pytest.raises(ps.PauliError) as e:
            ps.pauli_sum_upload_device(S, dv, dw, torch.tensor(re, dtype=torch.float64, device="cuda"),
                                      torch.tensor(im, dtype=torch.float64, device="cuda"))
        assert e.value.status == ps.PS_ERR_INVALID


def test_overflow_to_inf_is_reported_by_norm_trace_and_lanczos():
    n = 4
    big = 1.5e308
    H = ps.PauliSum.from_arrays(n, *I.single(n, "X", 1).arrays())
    O = ps.PauliSum.from_arrays(n, np.array([1], np.uint64), np.array([0], np.uint64), np.array([big]), np.zeros(1))
    C = ps.pauli_commutator(H, O)  # [X1, Z1] = -2i Y1: |coefficient| 3e308 overflows to Inf
    v, w, re, im = C.download()
    assert len(v) == 1 and np.isinf(im[0]) and re[0] == 0.0
    assert ps.pauli_norm(C) == float("inf")
    t = ps.pauli_trace_product(C, C)
    assert np.isnan(t.real) and np.isnan(t.imag)
    prev, cur = ps.PauliSum(n), ps.PauliSum.from_arrays(n, np.array([1], np.uint64), np.array([0], np.uint64),
                                                        np.array([big]), np.zeros(1))
    before = (_arrays(prev), _arrays(cur))
    with pytest.raises(ps.PauliError) as e:
        ps.pauli_lanczos_step(H, prev, cur, 0.0, None)
    assert e.value.status == ps.PS_ERR_NONFINITE
    assert _same(_arrays(prev), before[0]) and _same(_arrays(cur), before[1])
    # a finite start still works afterwards
    small = ps.PauliSum.from_arrays(n, np.array([1], np.uint64), np.array([0], np.uint64), np.array([1.0]), np.zeros(1))
    assert ps.pauli_lanczos_step(H, ps.PauliSum(n), small, 0.0, None) == 2.0


def test_download_into_too_small_capacity():
    n = 6
    rng = np.random.default_rng(2)
    v, w = I.random_strings(rng, n, 50)
    S = ps.PauliSum.from_arrays(n, v, w, rng.standard_normal(50), np.zeros(50))
    import ctypes
    lib = ps.load()
    buf = [np.zeros(10, np.uint64), np.zeros(10, np.uint64), np.zeros(10), np.zeros(10)]
    got = ctypes.c_int64()
    ptrs = [buf[0].ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), buf[1].ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
            buf[2].ctypes.data_as(ctypes.POINTER(ctypes.c_double)), buf[3].ctypes.data_as(ctypes.POINTER(ctypes.c_double))]
    st = lib.pauli_sum_download(S.handle, *ptrs, 10, ctypes.byref(got))
    assert st == ps.PS_ERR_CAPACITY and got.value == 50
    assert not any(b.any() for b in buf)  # nothing written


def test_scorer_wait_that_runs_out_returns_timeout():
    # the scorer's wait on its tensor-core products is bounded: with the products switched off
    # (a signal that never comes) the call returns PS_ERR_TIMEOUT and the library stays usable
    from oracle import mlp as omlp
    n = 20
    arr = I.random_sum(3, n, 700, kind="real")
    O = ps.PauliSum.from_arrays(n, *arr)  # storage order = upload order
    model = ps.PauliMLP(n, seed=4)
    ps.pauli_debug_mlp_wait(1, 1000)
    try:
        with pytest.raises(ps.PauliError) as e:
            ps.pauli_mlp_scores(model, O, 0.0)
        assert e.value.status == ps.PS_ERR_TIMEOUT
    finally:
        ps.pauli_debug_mlp_wait(0, 1 << 26)
    z = ps.pauli_mlp_logits(model, O).cpu().numpy().astype(np.float64)
    want, _ = omlp.forward(ps.pauli_mlp_get_params(model).astype(np.float64), omlp.features(*arr, n))
    assert np.linalg.norm(z - want) <= 2e-2 * max(np.linalg.norm(want), 1.0)
