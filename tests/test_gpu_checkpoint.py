"""Checkpoint / resume: a saved and reloaded sum continues bit for bit like the original."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2410_09654_gb300 import inputs as I

from gpu_util import assert_match

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as orc  # noqa: E402
from paper_2410_09654_gb300 import paulistr as ps  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ps.load(build_if_missing=True)


def test_roundtrip_values_meta_and_precision(tmp_path):
    n = 40
    arr = I.random_sum(3, n, 5000, kind="complex")
    S = ps.PauliSum.from_arrays(n, *arr)
    S.save(str(tmp_path / "a.ckp"), meta=[0.5, 3.0, 2.0, 1.9])
    T = ps.PauliSum(n)
    meta = T.load(str(tmp_path / "a.ckp"))
    assert list(meta) == [0.5, 3.0, 2.0, 1.9]
    assert_match(T.download(), orc.Op(n, *S.download()), exact=True, what="roundtrip")
    S.set_precision(ps.PS_COEF_F32)
    S.save(str(tmp_path / "b.ckp"))
    U = ps.PauliSum(n)
    assert len(U.load(str(tmp_path / "b.ckp"))) == 0
    assert U.precision() == ps.PS_COEF_F32
    assert_match(U.download(), orc.Op(n, *S.download()), exact=True, what="FP32 roundtrip")
    E = ps.PauliSum(n)
    E.save(str(tmp_path / "e.ckp"))
    assert len(ps.PauliSum.from_arrays(n, *arr).load(str(tmp_path / "e.ckp"))) == 0


def test_rk4_resume_is_bit_exact(tmp_path):
    n = 10
    H = ps.PauliSum.from_arrays(n, *I.tilted_ising_chain(n).arrays())
    pol = ps.policy(max_weight=6, cutoff=1e-10)
    A = ps.PauliSum.from_arrays(n, *I.single(n, "Z", 1).arrays())
    for _ in range(12):
        ps.pauli_rk4_step(H, A, 0.05, pol)
    B = ps.PauliSum.from_arrays(n, *I.single(n, "Z", 1).arrays())
    for _ in range(6):
        ps.pauli_rk4_step(H, B, 0.05, pol)
    B.save(str(tmp_path / "rk4.ckp"), meta=[6 * 0.05, 6])
    C = ps.PauliSum(n)
    t, step = C.load(str(tmp_path / "rk4.ckp"))
    assert step == 6 and t == 6 * 0.05
    for _ in range(6):
        ps.pauli_rk4_step(H, C, 0.05, pol)
    assert_match(C.download(), orc.Op(n, *A.download()), exact=True, what="resumed RK4")


def test_lanczos_resume_is_bit_exact(tmp_path):
    n = 16
    H = ps.PauliSum.from_arrays(n, *I.xxz_chain(n).arrays())
    pol = ps.policy(top_k=2000)
    prev, cur, b, bs = ps.PauliSum(n), ps.PauliSum.from_arrays(n, *I.uniform_sum(n, "X").arrays()), 0.0, []
    for _ in range(4):
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
        bs.append(b)
    prev.save(str(tmp_path / "p.ckp"))
    cur.save(str(tmp_path / "c.ckp"), meta=bs)
    for _ in range(4):
        b = ps.pauli_lanczos_step(H, prev, cur, b, pol)
        bs.append(b)
    p2, c2 = ps.PauliSum(n), ps.PauliSum(n)
    p2.load(str(tmp_path / "p.ckp"))
    hist = list(c2.load(str(tmp_path / "c.ckp")))
    b2 = hist[-1]
    for _ in range(4):
        b2 = ps.pauli_lanczos_step(H, p2, c2, b2, pol)
        hist.append(b2)
    assert hist == bs
    assert_match(c2.download(), orc.Op(n, *cur.download()), exact=True, what="resumed Lanczos")


def test_bad_files_are_errors(tmp_path):
    n = 12
    S = ps.PauliSum.from_arrays(n, *I.random_sum(5, n, 300, kind="real"))
    path = tmp_path / "s.ckp"
    S.save(str(path), meta=[1.0])
    raw = bytearray(path.read_bytes())
    T = ps.PauliSum(n)
    for name, data in (("flipped", raw[:100] + bytes([raw[100] ^ 1]) + raw[101:]), ("short", raw[:-9]),
                       ("magic", b"X" + raw[1:]), ("empty", b"")):
        bad = tmp_path / f"{name}.ckp"
        bad.write_bytes(bytes(data))
        with pytest.raises(ps.PauliError) as e:
            T.load(str(bad))
        assert e.value.status == ps.PS_ERR_IO, name
    with pytest.raises(ps.PauliError) as e:
        T.load(str(tmp_path / "missing.ckp"))
    assert e.value.status == ps.PS_ERR_IO
    with pytest.raises(ps.PauliError) as e:
        ps.PauliSum(n + 1).load(str(path))
    assert e.value.status == ps.PS_ERR_INVALID
    with pytest.raises(ps.PauliError) as e:
        S.save(str(tmp_path / "no_such_dir" / "x.ckp"))
    assert e.value.status == ps.PS_ERR_IO


def test_sort_by_hash_keeps_contents_and_results():
    n = 64
    Ha = I.xxz_chain(n).arrays()
    Oa = I.random_sum(8, n, 60000, kind="real", max_support=12)
    O = ps.PauliSum.from_arrays(n, *Oa)
    S = ps.PauliSum.from_arrays(n, *Oa).sort_by_hash()
    assert_match(S.download(), orc.Op(n, *O.download()), exact=True, what="contents")
    H = ps.PauliSum.from_arrays(n, *Ha)
    a = ps.pauli_commutator(H, O)
    b = ps.pauli_commutator(H, S)
    assert_match(b.download(), orc.Op(n, *a.download()), exact=True, what="commutator of the sorted operand")
    one = ps.PauliSum.from_arrays(n, *I.single(n, "X", 3).arrays()).sort_by_hash()
    assert len(one) == 1 and len(ps.PauliSum(n).sort_by_hash()) == 0
