"""Batched instances on the GPU: one instance-tagged sum evolved with per-instance H
coefficients and caps equals the oracle's RK4 step of every instance alone (bit-exact)."""
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


def _setup(n, n_inst, cap_fn, W=(0.5, 2.0, 5.0)):
    tbits = max(1, (n_inst - 1).bit_length())
    N = n + tbits
    Hs = [I.random_field_xxz_chain(n, W[b % len(W)], b).arrays() for b in range(n_inst)]
    hcoef = np.stack([h[2] for h in Hs])
    Hc = ps.PauliSum.from_arrays(N, Hs[0][0], Hs[0][1], np.ones(len(Hs[0][0])), np.zeros(len(Hs[0][0])))
    caps = np.array([cap_fn(b) for b in range(n_inst)], np.int64)
    B = ps.PauliBatch(Hc, hcoef, n, caps)
    return N, Hs, Hc, B, caps


def _tagged(arrs, n):
    v = np.concatenate([a[0] | (np.uint64(b) << np.uint64(n)) for b, a in enumerate(arrs)])
    w = np.concatenate([a[1] for a in arrs])
    re = np.concatenate([a[2] for a in arrs])
    im = np.concatenate([a[3] for a in arrs])
    return v, w, re, im


def _untag(arrays, n, n_inst):
    v, w, re, im = arrays
    tag = (v >> np.uint64(n)).astype(np.int64)
    low = v & np.uint64((1 << n) - 1)
    out = []
    for b in range(n_inst):
        m = tag == b
        o = np.lexsort((w[m], low[m]))
        out.append((low[m][o], w[m][o], re[m][o], im[m][o]))
    return out


@pytest.mark.parametrize("trim", [0, 1])
def test_batch_rk4_equals_each_instance_alone(trim):
    n, n_inst = 12, 20
    N, Hs, Hc, B, caps = _setup(n, n_inst, lambda b: 1 << (6 + b % 5))
    O0 = [I.single(n, "Z", 6).arrays() for _ in range(n_inst)]
    O = ps.PauliSum.from_arrays(N, *_tagged(O0, n))
    ref = [orc.Op(n, *o) for o in O0]
    Ho = [orc.Op(n, *h) for h in Hs]
    for step in range(6):
        ps.pauli_batch_rk4_step(B, Hc, O, 0.05, trim_stages=trim)
        ref = orc.batch_rk4_step(Ho, ref, 0.05, caps, trim_stages=trim)
        got = _untag(O.download(), n, n_inst)
        for b in range(n_inst):
            assert_match(got[b], ref[b], exact=True, what=f"step {step} instance {b}")
    counts = ps.pauli_batch_counts(B, O)
    assert list(counts) == [len(r) for r in ref]
    norms = ps.pauli_batch_norms(B, O)
    assert np.allclose(norms, [orc.norm(r) for r in ref], rtol=1e-14, atol=0)


def test_batch_uneven_instances_and_empty_ones():
    # instances of very different sizes, some empty, no caps
    n, n_inst = 10, 7
    N, Hs, Hc, B, caps = _setup(n, n_inst, lambda b: 0)
    O0 = [I.random_sum(30 + b, n, [0, 1, 50, 0, 400, 3, 2000][b], kind="real", max_support=5) for b in range(n_inst)]
    O = ps.PauliSum.from_arrays(N, *_tagged(O0, n))
    ps.pauli_batch_rk4_step(B, Hc, O, 0.02)
    got = _untag(O.download(), n, n_inst)
    for b in range(n_inst):
        want = orc.rk4_step(orc.Op(n, *Hs[b]), orc.Op(n, *O0[b]), 0.02)
        assert_match(got[b], want, exact=True, what=f"instance {b}")


def test_batch_truncate_per_instance_caps():
    n, n_inst = 14, 9
    N, Hs, Hc, B, caps = _setup(n, n_inst, lambda b: [1, 5, 100, 0, 7, 3000, 2, 64, 999][b])
    O0 = [I.random_sum(70 + b, n, 1000 + 300 * b, kind="real", dyadic=(b % 2 == 0)) for b in range(n_inst)]
    O = ps.PauliSum.from_arrays(N, *_tagged(O0, n))
    ps.pauli_batch_truncate(B, O)
    got = _untag(O.download(), n, n_inst)
    for b in range(n_inst):
        want = orc.truncate(orc.Op(n, *O0[b]), top_k=int(max(caps[b], 0)))
        assert_match(got[b], want, exact=True, what=f"instance {b}")


def test_batch_rejects_bad_tags_and_shapes():
    n, n_inst = 8, 5
    N, Hs, Hc, B, caps = _setup(n, n_inst, lambda b: 10)
    bad = I.single(N, "Z", n + 3).arrays()  # tag 4 is fine ...
    O = ps.PauliSum.from_arrays(N, *bad)
    ps.pauli_batch_rk4_step(B, Hc, O, 0.05)
    bad = I.single(N, "X", n + 1).arrays()  # ... but an X letter in the tag bits is not
    O = ps.PauliSum.from_arrays(N, *bad)
    with pytest.raises(ps.PauliError) as e:
        ps.pauli_batch_rk4_step(B, Hc, O, 0.05)
    assert e.value.status == ps.PS_ERR_INVALID
    with pytest.raises(ps.PauliError):
        ps.PauliBatch(Hc, np.zeros((n_inst, len(Hs[0][0]))), n + 2)  # tags would not fit below n_sites
    with pytest.raises(ps.PauliError):
        ps.PauliBatch(Hc, np.zeros((n_inst, len(Hs[0][0]))), n - 1)  # H has bits at the tag position


def test_batch_rk4_steps_equals_single_steps():
    """pauli_batch_rk4_steps(n) is n calls of pauli_batch_rk4_step; checked against the
    oracle's per-instance steps."""
    n, n_inst = 10, 9
    N, Hs, Hc, B, caps = _setup(n, n_inst, lambda b: 1 << (5 + b % 4))
    O0 = [I.single(n, "Z", 5).arrays() for _ in range(n_inst)]
    O = ps.PauliSum.from_arrays(N, *_tagged(O0, n))
    ps.pauli_batch_rk4_steps(B, Hc, O, 0.05, 4, trim_stages=1)
    ref = [orc.Op(n, *o) for o in O0]
    Ho = [orc.Op(n, *h) for h in Hs]
    for _ in range(4):
        ref = orc.batch_rk4_step(Ho, ref, 0.05, caps, trim_stages=1)
    got = _untag(O.download(), n, n_inst)
    for b in range(n_inst):
        assert_match(got[b], ref[b], exact=True, what=f"instance {b}")
    before = O.download()
    ps.pauli_batch_rk4_steps(B, Hc, O, 0.05, 0)  # zero steps: unchanged
    assert all(np.array_equal(x, y) for x, y in zip(O.download(), before))


def test_batch_truncate_all_ties_many_instances():
    # every coefficient equal: every rank is decided by the keys (~v, ~w), so the selection
    # runs past the |c|^2 digits through the listed candidates; instances of several sizes,
    # caps below, at and above their sizes
    n, n_inst = 16, 40
    N, Hs, Hc, B, caps = _setup(n, n_inst, lambda b: [3, 50, 400, 0, 1, 2000, 257][b % 7])
    O0 = []
    for b in range(n_inst):
        v, w, _re, _im = I.random_sum(500 + b, n, 200 + 37 * b, kind="real")
        O0.append((v, w, np.full(len(v), 0.5), np.zeros(len(v))))
    O = ps.PauliSum.from_arrays(N, *_tagged(O0, n))
    ps.pauli_batch_truncate(B, O)
    got = _untag(O.download(), n, n_inst)
    for b in range(n_inst):
        want = orc.truncate(orc.Op(n, *O0[b]), top_k=int(max(caps[b], 0)))
        assert_match(got[b], want, exact=True, what=f"instance {b}")
