"""Seeded, synthetic inputs: Hamiltonians and initial operators shaped like the
paper's workloads, plus random Pauli sums for parity tests.

This module only builds lists of strings and coefficients.  It holds none of
the method's arithmetic (no products, phases, sums or truncation), and it is
the one module that both the CUDA path's callers and the oracle's callers use
to make inputs.  Every generator returns four numpy arrays (v, w, re, im):
bit i-1 of v is the Z bit of site i, bit i-1 of w its X bit, and the
coefficient multiplies the Hermitian string (site letters I, X, Y, Z).

Models follow the paper's Hamiltonians: the XX chain (eq. XXmodel), the XXX
chain (eq. XXXmodel), the chaotic Ising-type chain (eq. CC), the 2D XXZ and
XZ+ZX lattices (eqs. 2dXXZ, 2dXZZX), and the field-tilted chain and random-field
XXZ chain used as synthetic benchmark workloads.
"""
from __future__ import annotations

import math

import numpy as np

_BITS = {"I": (0, 0), "X": (0, 1), "Z": (1, 0), "Y": (1, 1)}
MASK64 = (1 << 64) - 1


def string(*letters_sites) -> tuple[int, int]:
    """``string("X", 1, "Y", 2)`` -> (v, w) of X_1 Y_2 (sites are 1-indexed)."""
    v = w = 0
    it = iter(letters_sites)
    for letter, site in zip(it, it):
        zb, xb = _BITS[letter]
        v |= zb << (site - 1)
        w |= xb << (site - 1)
    return v, w


class SumBuilder:
    """Ordered list of (string, coefficient) terms; order is kept as added."""

    def __init__(self, n_sites: int):
        if not 1 <= n_sites <= 64:
            raise ValueError("n_sites must be in 1..64 (one 64-bit word per mask)")
        self.n = n_sites
        self.terms: list[tuple[int, int, complex]] = []

    def add(self, coef: complex, *letters_sites) -> "SumBuilder":
        v, w = string(*letters_sites)
        self.terms.append((v, w, complex(coef)))
        return self

    def arrays(self):
        v = np.array([t[0] for t in self.terms], dtype=np.uint64)
        w = np.array([t[1] for t in self.terms], dtype=np.uint64)
        re = np.array([t[2].real for t in self.terms], dtype=np.float64)
        im = np.array([t[2].imag for t in self.terms], dtype=np.float64)
        return v, w, re, im


# ----------------------------------------------------------------------------- chains
def xx_chain(n: int):
    """Open XX chain, eq. XXmodel: sum_j X_j X_{j+1} + Y_j Y_{j+1}."""
    b = SumBuilder(n)
    for j in range(1, n):
        b.add(1.0, "X", j, "X", j + 1)
        b.add(1.0, "Y", j, "Y", j + 1)
    return b


def xxz_chain(n: int, delta: float = 0.5):
    """Open XXZ chain: sum_j X_j X_{j+1} + Y_j Y_{j+1} + delta Z_j Z_{j+1} (3(n-1) strings)."""
    b = SumBuilder(n)
    for j in range(1, n):
        b.add(1.0, "X", j, "X", j + 1)
        b.add(1.0, "Y", j, "Y", j + 1)
        b.add(delta, "Z", j, "Z", j + 1)
    return b


def xxz_generator(n: int, delta: float = 0.5):
    """Translation generator H_0 of the periodic XXZ chain: X_1X_2 + Y_1Y_2 + delta Z_1Z_2
    (H = sum_i T_i(H_0) on a ring of n sites)."""
    b = SumBuilder(n)
    b.add(1.0, "X", 1, "X", 2)
    b.add(1.0, "Y", 1, "Y", 2)
    b.add(delta, "Z", 1, "Z", 2)
    return b


def tilted_ising_generator(n: int, jz: float = 1.0, hx: float = 1.05, hz: float = 0.5):
    """Translation generator of the periodic chain sum Z_iZ_{i+1} + hx X_i + hz Z_i."""
    b = SumBuilder(n)
    b.add(jz, "Z", 1, "Z", 2)
    b.add(hx, "X", 1)
    b.add(hz, "Z", 1)
    return b


def xxx_chain(n: int):
    """Open XXX chain, eq. XXXmodel."""
    return xxz_chain(n, 1.0)


def tilted_ising_chain(n: int, jz: float = 1.0, hx: float = 1.05, hz: float = 0.5):
    """Open chain sum Z_i Z_{i+1} + hx sum X_i + hz sum Z_i (3n-1 strings; a rotated
    form of the chaotic chain of eq. CC)."""
    b = SumBuilder(n)
    for j in range(1, n):
        b.add(jz, "Z", j, "Z", j + 1)
    for j in range(1, n + 1):
        b.add(hx, "X", j)
    for j in range(1, n + 1):
        b.add(hz, "Z", j)
    return b


def chaotic_ising_chain(n: int, hx: float = 0.5):
    """Eq. CC: sum X_i X_{i+1} - 1.05 Z_i + hx X_i (open)."""
    b = SumBuilder(n)
    for j in range(1, n):
        b.add(1.0, "X", j, "X", j + 1)
    for j in range(1, n + 1):
        b.add(-1.05, "Z", j)
        b.add(hx, "X", j)
    return b


def splitmix64(state: int) -> tuple[int, int]:
    """One step of the SplitMix64 generator (Steele, Lea, Flood 2014): (new state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def random_field_xxz_chain(n: int, W: float, instance: int, base_seed: int = 20241012):
    """Random-field XXZ (XXX) chain: sum X X + Y Y + Z Z + sum h_i Z_i, h_i ~ U[-W, W]
    from SplitMix64 seeded with base_seed + instance (top 53 bits -> [0, 1))."""
    b = SumBuilder(n)
    for j in range(1, n):
        b.add(1.0, "X", j, "X", j + 1)
        b.add(1.0, "Y", j, "Y", j + 1)
        b.add(1.0, "Z", j, "Z", j + 1)
    s = base_seed + instance
    for j in range(1, n + 1):
        s, r = splitmix64(s)
        u = (r >> 11) * (1.0 / (1 << 53))
        b.add(W * (2.0 * u - 1.0), "Z", j)
    return b


# ----------------------------------------------------------------------------- lattices
def lattice_site(r: int, c: int, cols: int) -> int:
    """1-indexed site of row r, column c (row-major)."""
    return (r - 1) * cols + c


def heisenberg_2d(rows: int, cols: int, jxy: float = 1.0, jz: float = 1.0):
    """Open square lattice, sum over bonds <ij> of X_i X_j + Y_i Y_j + jz Z_i Z_j
    (eq. 2dXXZ with jz = 1/2; Heisenberg with jz = 1).  Horizontal bonds first."""
    n = rows * cols
    b = SumBuilder(n)
    bonds = []
    for r in range(1, rows + 1):
        for c in range(1, cols):
            bonds.append((lattice_site(r, c, cols), lattice_site(r, c + 1, cols)))
    for r in range(1, rows):
        for c in range(1, cols + 1):
            bonds.append((lattice_site(r, c, cols), lattice_site(r + 1, c, cols)))
    for i, j in bonds:
        b.add(jxy, "X", i, "X", j)
        b.add(jxy, "Y", i, "Y", j)
        b.add(jz, "Z", i, "Z", j)
    return b


def xz_zx_2d(rows: int, cols: int):
    """Eq. 2dXZZX: sum_{xy} X_{x,y} Z_{x+1,y} + Z_{x,y} X_{x,y+1} (open)."""
    n = rows * cols
    b = SumBuilder(n)
    for r in range(1, rows + 1):
        for c in range(1, cols + 1):
            if r < rows:
                b.add(1.0, "X", lattice_site(r, c, cols), "Z", lattice_site(r + 1, c, cols))
            if c < cols:
                b.add(1.0, "Z", lattice_site(r, c, cols), "X", lattice_site(r, c + 1, cols))
    return b


# ----------------------------------------------------------------------------- operators
def single(n: int, letter: str, site: int, coef: complex = 1.0):
    return SumBuilder(n).add(coef, letter, site)


def uniform_sum(n: int, letter: str, coef: float | None = None):
    """sum_i letter_i with each coefficient ``coef`` (default 1/sqrt(n): unit norm)."""
    c = 1.0 / math.sqrt(n) if coef is None else coef
    b = SumBuilder(n)
    for j in range(1, n + 1):
        b.add(c, letter, j)
    return b


# ----------------------------------------------------------------------------- random sums
def random_strings(rng: np.random.Generator, n_sites: int, m: int, max_support: int | None = None,
                   unique: bool = True):
    """m random strings on n_sites; with max_support, each string lives on a random window
    of that many consecutive sites (local operators, like those the method produces)."""
    full = (1 << n_sites) - 1 if n_sites < 64 else MASK64
    out = []
    seen = set()
    tries = 0
    while len(out) < m:
        tries += 1
        if tries > 50 * m + 1000:
            raise ValueError("not enough distinct strings for the requested size")
        if max_support is None or max_support >= n_sites:
            v = int(rng.integers(0, 1 << 62, dtype=np.int64)) * 4 + int(rng.integers(0, 4))
            w = int(rng.integers(0, 1 << 62, dtype=np.int64)) * 4 + int(rng.integers(0, 4))
            v &= full
            w &= full
        else:
            start = int(rng.integers(0, n_sites - max_support + 1))
            win = ((1 << max_support) - 1) << start
            v = int(rng.integers(0, 1 << max_support)) << start
            w = int(rng.integers(0, 1 << max_support)) << start
            v &= win
            w &= win
        if unique:
            if (v, w) in seen:
                continue
            seen.add((v, w))
        out.append((v, w))
    v = np.array([s[0] for s in out], dtype=np.uint64)
    w = np.array([s[1] for s in out], dtype=np.uint64)
    return v, w


def random_sum(seed: int, n_sites: int, m: int, kind: str = "real", max_support: int | None = None,
               dyadic: bool = False):
    """Random Pauli sum of m distinct strings.  kind: 'real', 'imag' or 'complex'.
    dyadic: coefficients are small multiples of powers of two (sums stay exact)."""
    rng = np.random.default_rng(seed)
    v, w = random_strings(rng, n_sites, m, max_support)
    if dyadic:
        re = rng.integers(-8, 9, m).astype(np.float64) * 2.0 ** -rng.integers(0, 4, m)
        im = rng.integers(-8, 9, m).astype(np.float64) * 2.0 ** -rng.integers(0, 4, m)
    else:
        re = rng.standard_normal(m) * np.exp(rng.uniform(-6, 0, m))
        im = rng.standard_normal(m) * np.exp(rng.uniform(-6, 0, m))
    if kind == "real":
        im = np.zeros(m)
    elif kind == "imag":
        re = np.zeros(m)
    nz = (re != 0) | (im != 0)
    return v[nz], w[nz], re[nz], im[nz]
