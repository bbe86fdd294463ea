"""The seeded input generators: SplitMix64 against its published first outputs, and the
random-field chain's shape, field ranges and reproducibility (CPU only)."""
import numpy as np

from paper_2410_09654_gb300 import inputs as I


def test_splitmix64_published_sequence():
    # SplitMix64 from state 0 (Steele, Lea, Flood 2014; the generator seeding xoshiro):
    # first outputs 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4
    s, a = I.splitmix64(0)
    s, b = I.splitmix64(s)
    assert (a, b) == (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4)


def test_random_field_chain_shape_and_fields():
    n = 32
    for W, inst in ((0.5, 0), (2.0, 171), (5.0, 511)):
        v, w, re, im = I.random_field_xxz_chain(n, W, inst).arrays()
        assert len(v) == 3 * (n - 1) + n == 125
        assert not im.any()
        bonds, fields = re[: 3 * (n - 1)], re[3 * (n - 1):]
        assert np.all(bonds == 1.0)
        assert np.all(np.abs(fields) <= W) and len(set(fields.tolist())) == n
        # the string list is the same for every instance; only the fields differ
        v0, w0, re0, _ = I.random_field_xxz_chain(n, W, inst + 1).arrays()
        assert np.array_equal(v, v0) and np.array_equal(w, w0) and not np.array_equal(re, re0)
        assert np.array_equal(re, I.random_field_xxz_chain(n, W, inst).arrays()[2])
