"""FP32 arithmetic with compensated sums (precision PS_COEF_F32C) on the GPU, through the C
ABI, against the oracle of that arithmetic (oracle/f32c.py): commutators, linear
combinations, RK4 and Lanczos steps, bit for bit (the order of the terms and every FP32
rounding are defined, so the results are unique)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
from oracle import f32c
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


def dev(n, arrays):
    return ps.PauliSum.from_arrays(n, *arrays).set_precision(ps.PS_COEF_F32C)


def ref(n, arrays):
    return orc.round32(orc.Op(n, *arrays))


@pytest.mark.parametrize("n,mh,mo", [(10, 29, 400), (40, 60, 3000), (64, 150, 4000)])
def test_commutator_and_add(n, mh, mo):
    Ha = I.random_sum(21 + n, n, mh, kind="real", max_support=3)
    Oa = I.random_sum(22 + n, n, mo, kind="real", max_support=8)
    H, O = dev(n, Ha), dev(n, Oa)
    C = ps.PauliSum(n).set_precision(ps.PS_COEF_F32C)
    ps.pauli_commutator(H, O, C)
    Cr = f32c.commutator(ref(n, Ha), ref(n, Oa))
    assert_match(C.download(), Cr, what="[H,O] f32c")
    with pytest.raises(ps.PauliError) as e:  # a real sum plus the imaginary commutator: complex
        ps.pauli_add(O, -0.3, C, ps.PauliSum(n).set_precision(ps.PS_COEF_F32C))
    assert e.value.status == ps.PS_ERR_INVALID
    S2 = ps.PauliSum(n).set_precision(ps.PS_COEF_F32C)
    ps.pauli_add(O, 0.7, O.copy(), S2)
    assert_match(S2.download(), f32c.add(ref(n, Oa), 0.7, ref(n, Oa)), what="O + 0.7 O f32c")


def test_complex_merges_are_refused():
    n = 6
    Oa = I.random_sum(5, n, 50, kind="complex")
    O = dev(n, Oa)
    H = dev(n, I.tilted_ising_chain(n).arrays())
    with pytest.raises(ps.PauliError) as e:
        ps.pauli_commutator(H, O, ps.PauliSum(n).set_precision(ps.PS_COEF_F32C))
    assert e.value.status == ps.PS_ERR_INVALID


def test_rk4_chain_with_weight_and_cutoff():
    n = 10
    Ha = I.tilted_ising_chain(n).arrays()
    H, O = dev(n, Ha), dev(n, I.single(n, "Z", 1).arrays())
    Hr, Or = ref(n, Ha), ref(n, I.single(n, "Z", 1).arrays())
    pol = ps.policy(max_weight=6, cutoff=1e-10)
    for step in range(5):
        ps.pauli_rk4_step(H, O, 0.05, pol)
        Or = f32c.rk4_step(Hr, Or, 0.05, max_weight=6, cutoff=1e-10)
        assert_match(O.download(), Or, what=f"rk4 step {step}")


@pytest.mark.parametrize("rows,cols,cap", [(4, 4, 600), (8, 8, 250)])
def test_rk4_lattice_dissipation_trimmed(rows, cols, cap):
    # 4x4: 72 terms (six-word masks, full records); 8x8: 336 terms (512-bit masks, gathers)
    n = rows * cols
    Ha = I.heisenberg_2d(rows, cols).arrays()
    site = (rows // 2 - 1) * cols + cols // 2
    H, O = dev(n, Ha), dev(n, I.single(n, "Z", site).arrays())
    Hr, Or = ref(n, Ha), ref(n, I.single(n, "Z", site).arrays())
    pol = ps.policy(top_k=cap, gamma=0.1, trim_stages=1)
    for step in range(3):
        ps.pauli_rk4_step(H, O, 0.02, pol)
        Or = f32c.rk4_step(Hr, Or, 0.02, top_k=cap, gamma=0.1, trim_stages=1)
        assert_match(O.download(), Or, what=f"lattice {rows}x{cols} step {step}")


def test_lanczos_xxz():
    n = 12
    Ha = I.xxz_chain(n, 0.5).arrays()
    H = dev(n, Ha)
    prev, cur = ps.PauliSum(n).set_precision(ps.PS_COEF_F32C), dev(n, I.uniform_sum(n, "X").arrays())
    Hr = ref(n, Ha)
    rprev, rcur = orc.Op.empty(n), ref(n, I.uniform_sum(n, "X").arrays())
    b = rb = 0.0
    for step in range(6):
        b = ps.pauli_lanczos_step(H, prev, cur, b, ps.policy(top_k=500))
        rb, rn = f32c.lanczos_step(Hr, rprev, rcur, rb, top_k=500)
        rprev, rcur = rcur, rn
        assert b == rb, step
        assert_match(cur.download(), rcur, what=f"O_{step + 1}")
