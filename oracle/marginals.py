"""Median-of-means norm estimates, marginal probabilities and chain-rule sampling of
w output bits by norm estimation (oracle; test infrastructure only).

End of Sec. 4.3 of arXiv:1808.00128: the estimate of ||psi||^2 is made reliable by
taking K independent empirical means (each over L equatorial states) and their
median; the marginal of the bits on qubits q_1..q_w is P_w(x) = ||Pi psi||^2 /
||psi||^2 with Pi the product of the projectors (I + (-1)^{x_j} Z_{q_j})/2, a
stabilizer decomposition of Pi psi being the terms of psi pushed through the
projective gates of Sec. 4.1; the bits are then sampled one by one by the chain rule
P(x) = P_1(x_1) P_2(x_2 | x_1) ...

Readings taken here (the paper sketches the procedure without fixing them):
  * Group g of the K means uses the equatorial states l = g L .. g L + L - 1 of one
    draw stream; the median of an even number of means is the average of the two
    middle ones.
  * Step i (0-based) conditions on the bits already drawn by estimating both
    branches, p_b = ||Pi_{x_<i, b} psi||^2 for b = 0, 1, with the same equatorial
    states (stream seed_i = rand64(seed, 2^41 + i, 0)), and takes
    P(x_i = 1 | x_<i) = p_1 / (p_0 + p_1); x_i = 1 iff
    uniform(seed, 2^42 + i, 0) < p_1 / (p_0 + p_1), and x_i = 0 when p_0 + p_1 <= 0.
"""
from __future__ import annotations

import numpy as np

from . import estimators as E
from . import rng

STEP_STREAM = 1 << 41
DRAW_STREAM = 1 << 42


def median_of_means(etas, L: int, K: int) -> float:
    """Median of the K means of consecutive groups of L samples."""
    etas = np.asarray(etas, dtype=np.float64)
    if etas.size != L * K:
        raise ValueError("need L*K samples")
    means = etas.reshape(K, L).mean(axis=1)
    return float(np.median(means))


def project(terms, q: int, b: int):
    """Copies of the terms with (I + (-1)^b Z_q)/2 applied (Sec. 4.1 projective gates)."""
    out = []
    for t in terms:
        c = t.copy()
        c.apply_proj(q, b)
        out.append(c)
    return out


def norm_mom(terms, coefs, L: int, K: int, seed: int, As=None) -> float:
    """Median-of-means estimate of ||psi||^2 from L*K equatorial states of stream `seed`
    (or from the given list of A matrices, one group per K)."""
    n = terms[0].n
    if As is None:
        As = [E.draw_A(n, seed, l) for l in range(L * K)]
    return median_of_means([E.eta(terms, coefs, A) for A in As], L, K)


def marginal_sample(terms, coefs, qubits, L: int, K: int, seed: int, As=None):
    """Chain-rule sample of the bits on `qubits`.  Returns (bits, [(p0, p1) per step]).
    `As`, when given, replaces the equatorial draws of every step (exhaustive checks)."""
    n = terms[0].n
    bits, probs = [], []
    pref = list(terms)
    for i, q in enumerate(qubits):
        s_i = rng.rand64(seed, STEP_STREAM + i, 0)
        A_i = As if As is not None else [E.draw_A(n, s_i, l) for l in range(L * K)]
        branch = [project(pref, q, b) for b in (0, 1)]
        p = [norm_mom(branch[b], coefs, L, K, s_i, As=A_i) for b in (0, 1)]
        u = rng.uniform(seed, DRAW_STREAM + i, 0)
        tot = p[0] + p[1]
        x = 1 if (tot > 0 and u < p[1] / tot) else 0
        bits.append(x)
        probs.append((p[0], p[1]))
        pref = branch[x]
    return bits, probs
