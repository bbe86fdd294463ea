"""Parity at the benchmark's full size, in the launch configuration the benchmark times:
the Lanczos recursion on the open XXZ chain N=64 (189 strings), O_0 = sum X_i / 8, top 2^22
strings kept per step.  The GPU ramps the operator to the cap; then one step runs on the
GPU and the same step, from the downloaded state, in the oracle (about 8e8 string
products).  b_{n+1} and every kept string and coefficient must be bit-identical."""
from __future__ import annotations

import pytest

from paper_2410_09654_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as orc  # noqa: E402
from paper_2410_09654_gb300 import paulistr as ps  # noqa: E402

from gpu_util import assert_match  # noqa: E402

N = 64
CAP = 1 << 22


def test_lanczos_step_full_size_bit_exact():
    ps.load(build_if_missing=True)
    Ha = I.xxz_chain(N, 0.5).arrays()
    H = ps.PauliSum.from_arrays(N, *Ha)
    prev, cur = ps.PauliSum(N), ps.PauliSum.from_arrays(N, *I.uniform_sum(N, "X").arrays())
    pol = ps.policy(top_k=CAP)
    b = 0.0
    steps = 0
    while len(cur) < CAP or len(prev) < CAP:  # both operands at the cap, as in the timed steps
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
        steps += 1
        assert steps < 30
    rprev, rcur = orc.Op(N, *prev.download()), orc.Op(N, *cur.download())
    st_b = b
    b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
    merged = ps.pauli_last_merge_stats()
    rb, rnext = orc.lanczos_step(orc.Op(N, *Ha), rprev, rcur, st_b, top_k=CAP)
    assert b == rb, (b, rb)
    assert len(cur) == CAP
    assert merged["contributions"] > 5 * 10**7  # the full-size product count was exercised
    assert_match(cur.download(), rnext, what="full-size Lanczos step")
    assert_match(prev.download(), rcur, what="full-size Lanczos rotation")
