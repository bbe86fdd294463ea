"""Dense-matrix checker for tiny systems (N <= 6).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  This module builds Pauli
strings as explicit 2^N x 2^N Kronecker products of the textbook matrices
I, X, Y, Z and never uses the (v, w) phase formulas, so it pins them
independently.  Letter of site i (bit i-1): (v, w) = (0,0) I, (0,1) X,
(1,0) Z, (1,1) Y (v is the Z bit and w the X bit, paper's tau table).
"""
from __future__ import annotations

import numpy as np

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
LETTER = {(0, 0): I2, (0, 1): X, (1, 0): Z, (1, 1): Y}


def string_matrix(v: int, w: int, n: int) -> np.ndarray:
    """Kronecker product over sites 1..n (site 1 leftmost)."""
    m = np.ones((1, 1), dtype=complex)
    for i in range(n):
        m = np.kron(m, LETTER[((v >> i) & 1, (w >> i) & 1)])
    return m


def op_matrix(op, n: int) -> np.ndarray:
    d = 2 ** n
    m = np.zeros((d, d), dtype=complex)
    for v, w, re, im in zip(op.v, op.w, op.re, op.im):
        m += complex(re, im) * string_matrix(int(v), int(w), n)
    return m


def decompose(m: np.ndarray, n: int) -> dict:
    """Coefficients c_s = Tr(P_s M)/2^N (the Hermitian strings are trace-orthonormal)."""
    out = {}
    d = 2 ** n
    for v in range(2 ** n):
        for w in range(2 ** n):
            c = np.trace(string_matrix(v, w, n) @ m) / d
            if abs(c) > 0:
                out[(v, w)] = complex(c)
    return out


def commutator(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return a @ b - b @ a


def rk4_dense(h: np.ndarray, o: np.ndarray, dt: float) -> np.ndarray:
    """Classical RK4 for dO/dt = i[H, O] on matrices (same stage formula as the oracle)."""
    f = lambda x: 1j * commutator(h, x)
    k1 = f(o)
    k2 = f(o + (dt / 2) * k1)
    k3 = f(o + (dt / 2) * k2)
    k4 = f(o + dt * k3)
    return o + (dt / 6) * (k1 + 2 * k2 + 2 * k3 + k4)


def heisenberg_exact(h: np.ndarray, o: np.ndarray, t: float) -> np.ndarray:
    """O(t) = e^{iHt} O e^{-iHt}, the exact solution of dO/dt = i[H, O]."""
    ev, u = np.linalg.eigh(h)
    ph = np.exp(1j * ev * t)
    ut = (u * ph) @ u.conj().T
    return ut @ o @ ut.conj().T


def lanczos_dense(h: np.ndarray, o0: np.ndarray, n_steps: int, n: int) -> list[float]:
    """Lanczos on the Liouvillian L = [H, .] with <A,B> = Tr(A^dag B)/2^N, no truncation."""
    d = 2 ** n
    ip = lambda a, b: np.trace(a.conj().T @ b) / d
    nrm = lambda a: float(np.sqrt(max(ip(a, a).real, 0.0)))
    bs = []
    a = commutator(h, o0)
    b = nrm(a)
    bs.append(b)
    prev, cur = o0, a / b
    for _ in range(2, n_steps + 1):
        a = commutator(h, cur) - b * prev
        b = nrm(a)
        bs.append(b)
        if b < 1e-12:
            break
        prev, cur = cur, a / b
    return bs
