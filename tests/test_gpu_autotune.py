"""The merge geometry autotuner: every candidate geometry gives the oracle's result bit for
bit, and tuning picks one of the candidates for the size class."""
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
    ps.pauli_autotune_reset()


@pytest.mark.parametrize("bt,q", [(64, 64), (1024, 1024), (4096, 1536), (65536, 4096), (2048, 2000)])
def test_each_geometry_is_exact(bt, q):
    n = 40
    Ha = I.random_sum(3, n, 120, kind="real", max_support=5)
    Oa = I.random_sum(4, n, 30000, kind="real", max_support=9)
    ps.pauli_merge_geometry_fix(bt, q)
    try:
        got = ps.pauli_commutator(ps.PauliSum.from_arrays(n, *Ha), ps.PauliSum.from_arrays(n, *Oa))
        # a wide-geometry merge (|H| + sources beyond 256) and a source merge too
        Hw = I.random_sum(5, n, 300, kind="real", max_support=4)
        gw = ps.pauli_commutator(ps.PauliSum.from_arrays(n, *Hw), ps.PauliSum.from_arrays(n, *Oa))
        ga = ps.pauli_add(ps.PauliSum.from_arrays(n, *Oa), 0.5, got)
    finally:
        ps.pauli_autotune_reset()
    want = orc.commutator(orc.Op(n, *Ha), orc.Op(n, *Oa))
    assert_match(got.download(), want, exact=True, what=f"geometry {bt},{q}")
    assert_match(gw.download(), orc.commutator(orc.Op(n, *Hw), orc.Op(n, *Oa)), exact=True, what="wide")
    assert_match(ga.download(), orc.axpy(orc.Op(n, *Oa), 0.5, want), exact=True, what="add")


def test_autotune_picks_a_candidate_and_keeps_results():
    n = 48
    H = ps.PauliSum.from_arrays(n, *I.tilted_ising_chain(n).arrays())
    Oa = I.random_sum(8, n, 50000, kind="real", max_support=10)
    O = ps.PauliSum.from_arrays(n, *Oa)
    r = ps.pauli_autotune_commutator(H, O, reps=2)
    assert r["bin_target"] in (1024, 2048, 4096) and r["quota"] in (1024, 1536)
    assert 0 < r["best_ms"] <= r["default_ms"]
    got = ps.pauli_commutator(H, O)  # runs in the tuned geometry
    want = orc.commutator(orc.Op(n, *I.tilted_ising_chain(n).arrays()), orc.Op(n, *Oa))
    assert_match(got.download(), want, exact=True, what="tuned")
    with pytest.raises(ps.PauliError):
        ps.pauli_merge_geometry_fix(10, 1536)


@pytest.mark.parametrize("m", [8000, 9000, 300])
def test_plan_boundary_bins(m):
    # 120 terms x m strings at 64 entries per bin: 2^14 bins for m = 8000 (the largest merge
    # planned in one block, 16 bins per thread), 2^15 for m = 9000 (the device-wide plan),
    # a few hundred bins for m = 300; the results do not depend on the path
    n = 40
    Ha = I.random_sum(13, n, 120, kind="real", max_support=5)
    Oa = I.random_sum(14, n, m, kind="real", max_support=9)
    ps.pauli_merge_geometry_fix(64, 64)
    try:
        got = ps.pauli_commutator(ps.PauliSum.from_arrays(n, *Ha), ps.PauliSum.from_arrays(n, *Oa))
        ga = ps.pauli_add(ps.PauliSum.from_arrays(n, *Oa), -0.25, got)
    finally:
        ps.pauli_autotune_reset()
    want = orc.commutator(orc.Op(n, *Ha), orc.Op(n, *Oa))
    assert_match(got.download(), want, exact=True, what=f"plan m={m}")
    assert_match(ga.download(), orc.axpy(orc.Op(n, *Oa), -0.25, want), exact=True, what=f"add m={m}")
