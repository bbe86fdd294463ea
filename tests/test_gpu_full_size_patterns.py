"""Parity of the three benchmark patterns at the sizes the benchmark runs them:
the 512 batched disorder realisations (N=32, caps 2^8..2^14 per instance) checked on sampled
instances against the oracle run alone from the same state; the learned truncation at cap
2^18 on the N=48 chain checked on a sample of the real candidates (features and logits to
BF16 tolerance) and on its kept set (exactly the top-k by the library's rank values); the
FP32 lattice workload checked for FP32 values and its distance from the FP64 run."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2410_09654_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as orc  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from paper_2410_09654_gb300 import paulistr as ps  # noqa: E402

from gpu_util import assert_match  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ps.load(build_if_missing=True)


def _instance(arrays, b, shift):
    v, w, re, im = arrays
    tag = (v >> np.uint64(shift)).astype(np.int64)
    m = tag == b
    return v[m] & np.uint64((1 << shift) - 1), w[m], re[m], im[m]


def test_batched_realisations_full_size_sampled_instances():
    n, shift, n_inst = 32, 32, 512
    N = shift + 9
    W = [0.5 if b <= 170 else (2.0 if b <= 341 else 5.0) for b in range(n_inst)]
    Hs = [I.random_field_xxz_chain(n, W[b], b).arrays() for b in range(n_inst)]
    caps = np.array([1 << (8 + b % 7) for b in range(n_inst)], np.int64)
    Hc = ps.PauliSum.from_arrays(N, Hs[0][0], Hs[0][1], np.ones(len(Hs[0][0])), np.zeros(len(Hs[0][0])))
    B = ps.PauliBatch(Hc, np.stack([h[2] for h in Hs]), shift, caps)
    z = I.single(n, "Z", 16).arrays()
    v = np.array([int(z[0][0]) | (b << shift) for b in range(n_inst)], np.uint64)
    O = ps.PauliSum.from_arrays(N, v, np.zeros(n_inst, np.uint64), np.ones(n_inst), np.zeros(n_inst))
    for _ in range(12):
        ps.pauli_batch_rk4_step(B, Hc, O, 0.05, trim_stages=1)
    before = O.download()
    ps.pauli_batch_rk4_step(B, Hc, O, 0.05, trim_stages=1)
    after = O.download()
    for b in (6, 13, 200, 503):  # caps 2^14, 2^14, 2^12, 2^14; three disorder strengths
        start = orc.Op(n, *_instance(before, b, shift))
        assert len(start) == caps[b]
        want = orc.rk4_step(orc.Op(n, *Hs[b]), start, 0.05, top_k=int(caps[b]), trim_stages=1)
        assert_match(_instance(after, b, shift), want, exact=True, what=f"instance {b}")


def test_learned_truncation_full_size_sampled():
    n = 48
    H = ps.PauliSum.from_arrays(n, *I.tilted_ising_chain(n).arrays())
    O = ps.PauliSum.from_arrays(n, *I.single(n, "Z", 24).arrays())
    pol = ps.policy(top_k=1 << 18, trim_stages=1)
    model = ps.PauliMLP(n, seed=4)
    C = ps.PauliSum(n)
    for _ in range(40):
        ps.pauli_rk4_step_mlp(H, O, 0.05, pol, model=model, cand_out=C)
    assert len(O) == 1 << 18 and len(C) > len(O)
    # the kept set is the top 2^18 of the candidates by the library's rank values
    rank = ps.pauli_mlp_scores(model, C, 0.0)
    m = len(C)
    import ctypes
    t = [torch.empty(m, dtype=dt, device="cuda") for dt in (torch.int64, torch.int64, torch.float64, torch.float64)]
    got = ctypes.c_int64()
    ps._check(ps.load().pauli_sum_download_device(C.handle, *[ctypes.c_void_p(x.data_ptr()) for x in t], m,
                                                   ctypes.byref(got)), "download_device")
    cv = t[0].cpu().numpy().view(np.uint64)
    cw = t[1].cpu().numpy().view(np.uint64)
    r = rank.cpu().numpy()
    order = np.lexsort((cw, cv, -r))  # rank descending, then v, then w ascending
    want = set(zip(cv[order[: 1 << 18]].tolist(), cw[order[: 1 << 18]].tolist()))
    ov, ow, _, _ = O.download()
    assert set(zip(ov.tolist(), ow.tolist())) == want
    # features and logits of a sample of the candidates against the oracle
    p = ps.pauli_mlp_get_params(model).astype(np.float64)
    idx = np.random.default_rng(0).choice(m, 3000, replace=False)
    cre = t[2].cpu().numpy()
    cim = t[3].cpu().numpy()
    S = ps.PauliSum.from_arrays(n, cv[idx], cw[idx], cre[idx], cim[idx])
    z = ps.pauli_mlp_logits(model, S).cpu().numpy().astype(np.float64)
    zo, _ = omlp.forward(p, omlp.features(cv[idx], cw[idx], cre[idx], cim[idx], n))
    assert np.linalg.norm(z - zo) / np.linalg.norm(zo) < 2e-2


def test_fp32_lattice_workload_stays_fp32_and_close():
    rows = cols = 8
    N = 64
    Ha = I.heisenberg_2d(rows, cols).arrays()
    Oa = I.single(N, "Z", 28).arrays()
    pol = ps.policy(top_k=1 << 20, gamma=0.1, trim_stages=1)
    runs = {}
    for prec in (ps.PS_COEF_F64, ps.PS_COEF_F32):
        H = ps.PauliSum.from_arrays(N, *Ha).set_precision(prec)
        O = ps.PauliSum.from_arrays(N, *Oa).set_precision(prec)
        for _ in range(14):
            ps.pauli_rk4_step(H, O, 0.02, pol)
        runs[prec] = O.download()
    a, b = runs[ps.PS_COEF_F32], runs[ps.PS_COEF_F64]
    assert len(a[0]) == 1 << 20
    assert np.array_equal(a[2], a[2].astype(np.float32).astype(np.float64))
    da = dict(zip(zip(a[0].tolist(), a[1].tolist()), a[2]))
    db = dict(zip(zip(b[0].tolist(), b[1].tolist()), b[2]))
    common = set(da) & set(db)
    assert len(common) > 0.99 * len(db)  # the kept sets differ only near the cut
    err = np.sqrt(sum((da[k] - db[k]) ** 2 for k in common))
    nrm = np.sqrt(sum(db[k] ** 2 for k in common))
    # each step rounds about ten stored results (~6e-8 each), but at the cap the rounding also
    # changes which near-tied strings the top-k keeps, and the strings dropped differently feed
    # the next steps: measured 8.8e-5 after 14 steps (pure rounding without a cap is pinned in
    # tests/test_f32_oracle.py)
    assert err < 5e-4 * nrm, err / nrm
