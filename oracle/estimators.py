"""Amplitudes, norm estimation and Metropolis chains (oracle; test only).

Sec. 4.2 ("Heuristic Metropolis simulator") and Sec. 4.3 ("Fast norm
estimation") of arXiv:1808.00128, for psi = sum_alpha b_alpha phi_alpha with
every phi_alpha a CH-form (oracle.chform.CHForm).  All arithmetic is FP64 or
exact integer.

Readings taken here:
  * Lemma (Inner Product) gives <phi|phi_A> for omega = 1; for a term with
    prefactor omega, <phi_A|omega phi> = omega * conj(<phi|phi_A>).
  * K = G^T (A + J) G is formed over the integers, then reduced (diagonal
    mod 4, off-diagonal mod 2), as in the proof of Lemma (Inner Product).
  * A in M_n is drawn from rng stream (seed, l): word 0 gives the low bits of
    diag(A), word 1 the high bits, and the strict upper triangle follows in
    row-major order from word 2 on (pair index k -> word 2 + k//64, bit k%64).
  * Metropolis (Sec. 4.2): step t of chain c takes j = floor(r * n / 2^32)
    with r the high 32 bits of rand64(seed, c, 2t), and the uniform
    rng.uniform(seed, c, 2t+1) for the acceptance test.  A chain at P(x) = 0
    accepts every move (P(y) >= P(x)), the literal rule.
"""
from __future__ import annotations

import math

import numpy as np

from . import rng
from .chform import CHForm, bit, popcount
from .expsum import expsum


# ------------------------------ amplitudes -------------------------------------------
def amplitude(terms, coefs, x: int) -> complex:
    """<x|psi> = sum_alpha b_alpha <x|phi_alpha>  (Eq. (amplitude1) per term)."""
    return complex(sum(b * t.amplitude(x) for t, b in zip(terms, coefs)))


def probability(terms, coefs, x: int) -> float:
    return abs(amplitude(terms, coefs, x)) ** 2


# ------------------------------ equatorial states ------------------------------------
def draw_A(n: int, seed: int, l: int) -> np.ndarray:
    """A_l in M_n as an integer matrix (diagonal 0..3, off-diagonal 0/1)."""
    A = np.zeros((n, n), dtype=np.int64)
    w0, w1 = rng.rand64(seed, l, 0), rng.rand64(seed, l, 1)
    for a in range(n):
        A[a, a] = bit(w0, a) + 2 * bit(w1, a)
    k = 0
    for a in range(n):
        for b in range(a + 1, n):
            word = rng.rand64(seed, l, 2 + k // 64)
            A[a, b] = A[b, a] = bit(word, k % 64)
            k += 1
    return A


def _bits_vec(x: int, n: int) -> np.ndarray:
    return np.array([bit(x, j) for j in range(n)], dtype=np.int64)


def _mat(rows, n) -> np.ndarray:
    return np.array([[bit(r, j) for j in range(n)] for r in rows], dtype=np.int64)


def inner_equatorial(ch: CHForm, A: np.ndarray) -> complex:
    """<phi|phi_A> for the omega = 1 part of `ch` (Lemma (Inner Product),
    Eq. (inner_explicit)), with Z(B) from Lemma (Exponential Sum)."""
    n = ch.n
    sKs, sv, nvars, re, im = inner_equatorial_parts(ch, A)
    return (2.0 ** (-(n + nvars) / 2)) * (1j ** sKs) * ((-1) ** sv) * complex(re, im)


def inner_equatorial_parts(ch: CHForm, A: np.ndarray):
    """The exact ingredients of <phi|phi_A> = 2^{-(n+|v|)/2} i^{sKs} (-1)^{s.v} Z(B)
    (Lemma (Inner Product)): (sKs mod 4, s.v mod 2, |v|, Re Z(B), Im Z(B))."""
    n = ch.n
    G, F, M = _mat(ch.G, n), _mat(ch.F, n), _mat(ch.M, n)
    # J in M_n: diag(J) = gamma, J_ab = (M F^T)_ab mod 2 for a != b
    J = (M @ F.T) % 2
    np.fill_diagonal(J, np.array(ch.gamma, dtype=np.int64))
    K = G.T @ (A + J) @ G                      # over the integers
    s = _bits_vec(ch.s, n)
    v = _bits_vec(ch.v, n)
    sKs = int(s @ K @ s) % 4
    lin = (s + s @ K) % 2                      # s + sK, only its parity enters 2 x (.)^T
    Bfull = K.copy()
    Bfull[np.diag_indices(n)] += 2 * lin
    idx = [j for j in range(n) if v[j]]
    B = [[int(Bfull[a, b]) % (4 if a == b else 2) for b in idx] for a in idx]
    re, im = expsum(B)
    sv = int(s @ v) % 2
    return sKs, sv, len(idx), re, im


def overlap_A(terms, coefs, A: np.ndarray) -> complex:
    """<phi_A|psi> = sum_alpha b_alpha omega_alpha conj(<phi'_alpha|phi_A>)."""
    tot = 0j
    for t, b in zip(terms, coefs):
        if t.zero:
            continue
        tot += b * t.omega() * inner_equatorial(t, A).conjugate()
    return tot


def eta(terms, coefs, A: np.ndarray) -> float:
    """eta_A = 2^n |<phi_A|psi>|^2  (Eq. (xi), Lemma (Norm Estimation))."""
    n = terms[0].n
    return (2.0 ** n) * abs(overlap_A(terms, coefs, A)) ** 2


def norm_estimate(terms, coefs, L: int, seed: int):
    """Empirical mean of eta over A_1..A_L (Sec. 4.3).  Returns (etas, mean)."""
    n = terms[0].n
    etas = [eta(terms, coefs, draw_A(n, seed, l)) for l in range(L)]
    return etas, float(np.mean(etas))


def all_equatorial(n: int):
    """Every A in M_n (for exhaustive checks at n <= 3)."""
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    for diag in range(4 ** n):
        for off in range(1 << len(pairs)):
            A = np.zeros((n, n), dtype=np.int64)
            for a in range(n):
                A[a, a] = (diag >> (2 * a)) & 3
            for k, (a, b) in enumerate(pairs):
                A[a, b] = A[b, a] = (off >> k) & 1
            yield A


# ------------------------------ Metropolis -------------------------------------------
def metropolis_draws(n: int, seed: int, chain: int, step: int):
    """(j, r) for step `step` of chain `chain`."""
    r1 = rng.rand64(seed, chain, 2 * step)
    j = ((r1 >> 32) * n) >> 32
    r = rng.uniform(seed, chain, 2 * step + 1)
    return j, r


def metropolis_step(terms, coefs, x: int, px: float, n: int, seed: int, chain: int, step: int):
    """One Metropolis step x -> x' (Sec. 4.2).  Returns (x', P(x'), accepted, ratio, r)."""
    j, r = metropolis_draws(n, seed, chain, step)
    y = x ^ (1 << j)
    py = probability(terms, coefs, y)
    if py >= px:
        return y, py, True, math.inf if px == 0 else py / px, r
    ratio = py / px
    if r < ratio:
        return y, py, True, ratio, r
    return x, px, False, ratio, r
