"""Dense state-vector simulator (oracle ground truth; test infrastructure only).

Basis index x holds qubit j in bit j.  Gates are the textbook matrices; this is
the reference every CH-form result is pinned to at small n.
"""
from __future__ import annotations

import numpy as np

SQ2 = 1 / np.sqrt(2.0)


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def _idx(n):
    return np.arange(1 << n, dtype=np.int64)


def apply_1q(psi: np.ndarray, n: int, q: int, U) -> np.ndarray:
    """Apply a 2x2 matrix U to qubit q."""
    x = _idx(n)
    b = (x >> q) & 1
    partner = x ^ (1 << q)
    out = np.empty_like(psi)
    # out[x] = sum_c U[b(x), c] psi[x with bit q = c]
    x0 = np.where(b == 0, x, partner)
    x1 = np.where(b == 0, partner, x)
    out = np.where(b == 0, U[0][0] * psi[x0] + U[0][1] * psi[x1],
                   U[1][0] * psi[x0] + U[1][1] * psi[x1])
    return out


def apply_gate(psi: np.ndarray, n: int, g) -> np.ndarray:
    name = g[0]
    x = _idx(n)
    if name == "H":
        return apply_1q(psi, n, g[1], ((SQ2, SQ2), (SQ2, -SQ2)))
    if name == "X":
        return psi[x ^ (1 << g[1])]
    if name in ("S", "SDG", "Z", "T", "TDG"):
        ph = {"S": 1j, "SDG": -1j, "Z": -1.0, "T": np.exp(1j * np.pi / 4),
              "TDG": np.exp(-1j * np.pi / 4)}[name]
        b = (x >> g[1]) & 1
        return psi * np.where(b == 1, ph, 1.0)
    if name == "RZ":
        theta = g[2]
        b = (x >> g[1]) & 1
        return psi * np.where(b == 1, np.exp(1j * theta / 2), np.exp(-1j * theta / 2))
    if name == "CZ":
        b = ((x >> g[1]) & 1) & ((x >> g[2]) & 1)
        return psi * np.where(b == 1, -1.0, 1.0)
    if name == "CCZ":
        b = ((x >> g[1]) & 1) & ((x >> g[2]) & 1) & ((x >> g[3]) & 1)
        return psi * np.where(b == 1, -1.0, 1.0)
    if name == "CX":
        c, t = g[1], g[2]
        src = np.where(((x >> c) & 1) == 1, x ^ (1 << t), x)
        return psi[src]
    if name in ("P0", "P1"):
        want = 0 if name == "P0" else 1
        b = (x >> g[1]) & 1
        return psi * (b == want)
    raise ValueError(f"unknown gate {g}")


def run(n: int, ops, psi: np.ndarray | None = None) -> np.ndarray:
    psi = zero_state(n) if psi is None else psi.copy()
    for g in ops:
        psi = apply_gate(psi, n, g)
    return psi


def gate_matrix(n: int, ops) -> np.ndarray:
    """Full 2^n x 2^n matrix of a gate list (small n only)."""
    dim = 1 << n
    out = np.zeros((dim, dim), dtype=np.complex128)
    for col in range(dim):
        e = np.zeros(dim, dtype=np.complex128)
        e[col] = 1.0
        out[:, col] = run(n, ops, e)
    return out


def equatorial_state(n: int, A: np.ndarray) -> np.ndarray:
    """phi_A = 2^{-n/2} sum_x i^{x A x^T} |x> (Eq. (eqa1)); A integer n x n."""
    x = _idx(n)
    bits = ((x[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)
    q = np.einsum("xa,ab,xb->x", bits, A.astype(np.int64), bits) % 4
    return (1j ** q) * 2.0 ** (-n / 2)
