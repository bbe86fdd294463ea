"""FP32 coefficients on the GPU against the oracle's FP32 compositions (bit-exact: both
round the same FP64 results once to FP32), and the mode's bookkeeping."""
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

F32 = ps.PS_COEF_F32


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ps.load(build_if_missing=True)


def f32sum(n, arrays):
    return ps.PauliSum.from_arrays(n, *arrays).set_precision(F32)


def r32(n, arrays):
    return orc.round32(orc.Op(n, *arrays))


def test_set_precision_rounds_and_drops_underflow():
    n = 6
    arr = (np.array([1, 2, 3], np.uint64), np.array([0, 1, 2], np.uint64), np.array([0.1, 1e-50, 2.0]),
           np.array([1.0 / 3.0, 0.0, 0.0]))
    S = ps.PauliSum.from_arrays(n, *arr)
    assert S.precision() == ps.PS_COEF_F64
    S.set_precision(F32)
    assert S.precision() == F32
    assert_match(S.download(), r32(n, arr), exact=True, what="set_precision")
    S.upload(*arr)  # uploads into an FP32 sum are rounded too
    assert_match(S.download(), r32(n, arr), exact=True, what="upload")
    C = S.copy()
    assert C.precision() == F32


@pytest.mark.parametrize("kind,nH,m", [("real", 40, 20000), ("complex", 60, 5000), ("real", 300, 3000)])
def test_commutator_f32(kind, nH, m):
    n = 40
    Ha = I.random_sum(1 + nH, n, nH, kind=kind, max_support=6)
    Oa = I.random_sum(2 + m, n, m, kind=kind, max_support=10)
    H, O = f32sum(n, Ha), f32sum(n, Oa)
    out = ps.PauliSum(n).set_precision(F32)
    ps.pauli_commutator(H, O, out)
    want = orc.commutator_f32(r32(n, Ha), r32(n, Oa))
    assert_match(out.download(), want, exact=True, what="FP32 commutator")


def test_rk4_f32_chain_weight_and_cutoff():
    n = 10
    Ha = I.tilted_ising_chain(n).arrays()
    H, O = f32sum(n, Ha), f32sum(n, I.single(n, "Z", 1).arrays())
    Ho, ref = r32(n, Ha), r32(n, I.single(n, "Z", 1).arrays())
    pol = ps.policy(max_weight=6, cutoff=1e-10)
    for step in range(12):
        ps.pauli_rk4_step(H, O, 0.05, pol)
        ref = orc.rk4_step_f32(Ho, ref, 0.05, max_weight=6, cutoff=1e-10)
        assert_match(O.download(), ref, exact=True, what=f"step {step}")


def test_rk4_f32_lattice_dissipation_trimmed_stages():
    Ha = I.heisenberg_2d(4, 4).arrays()
    n = 16
    H, O = f32sum(n, Ha), f32sum(n, I.single(n, "Z", 6).arrays())
    Ho, ref = r32(n, Ha), r32(n, I.single(n, "Z", 6).arrays())
    pol = ps.policy(top_k=1500, gamma=0.1, trim_stages=1)
    for step in range(6):
        ps.pauli_rk4_step(H, O, 0.02, pol)
        ref = orc.rk4_step_f32(Ho, ref, 0.02, top_k=1500, gamma=0.1, trim_stages=1)
        assert_match(O.download(), ref, exact=True, what=f"step {step}")


def test_lanczos_f32_xxz():
    n = 16
    Ha = I.xxz_chain(n).arrays()
    H = f32sum(n, Ha)
    prev, cur = ps.PauliSum(n).set_precision(F32), f32sum(n, I.uniform_sum(n, "X").arrays())
    Ho = r32(n, Ha)
    oprev, ocur = orc.Op.empty(n), r32(n, I.uniform_sum(n, "X").arrays())
    b = bo = 0.0
    for step in range(8):
        b = ps.pauli_lanczos_step(H, prev, cur, b, ps.policy(top_k=3000))
        bo, nxt = orc.lanczos_step_f32(Ho, oprev, ocur, bo, top_k=3000)
        oprev, ocur = ocur, nxt
        assert b == bo, (step, b, bo)
        assert_match(cur.download(), ocur, exact=True, what=f"O_{step + 1}")


def test_f32_equals_f64_on_dyadic_data():
    n = 12
    Ha = I.random_sum(5, n, 30, kind="real", dyadic=True)
    Oa = I.random_sum(6, n, 400, kind="real", dyadic=True)
    a = ps.PauliSum(n).set_precision(F32)
    ps.pauli_commutator(f32sum(n, Ha), f32sum(n, Oa), a)
    b = ps.pauli_commutator(ps.PauliSum.from_arrays(n, *Ha), ps.PauliSum.from_arrays(n, *Oa))
    assert_match(a.download(), orc.Op(n, *b.download()), exact=True, what="dyadic")
