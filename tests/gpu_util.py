"""Helpers for the GPU parity tests: compare a device sum with an oracle sum."""
from __future__ import annotations

import numpy as np

# FP64 tolerance: coefficients must agree to 1e-12 relative (per coefficient).  The CUDA
# path reproduces the oracle's rounding order, so the tests also require bit equality
# where stated (exact=True).
REL_TOL = 1e-12


def assert_match(gpu_arrays, ref, exact: bool = True, what: str = ""):
    v, w, re, im = gpu_arrays
    assert len(v) == len(ref.v), f"{what}: size {len(v)} != oracle {len(ref.v)}"
    assert np.array_equal(v, ref.v) and np.array_equal(w, ref.w), f"{what}: string sets differ"
    g = re + 1j * im
    r = ref.re + 1j * ref.im
    err = np.abs(g - r)
    bad = err > REL_TOL * np.abs(r)
    assert not bad.any(), f"{what}: {int(bad.sum())} coefficients beyond 1e-12 relative (max {float((err / np.abs(r)).max())})"
    if exact:
        assert np.array_equal(re, ref.re) and np.array_equal(im, ref.im), \
            f"{what}: not bit-identical ({int((re != ref.re).sum() + (im != ref.im).sum())} differ)"
