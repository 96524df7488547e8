"""Pins for the oracle's median-of-means estimate and chain-rule marginal sampler
(end of Sec. 4.3): the median of means by hand, the projected decomposition against
dense projectors, exact marginals (equatorial average over all of M_n, n <= 3)
against the dense state vector, and chain-rule sample frequencies against the dense
marginal distribution."""
import random

import numpy as np
import pytest

from oracle import dense
from oracle import estimators as E
from oracle import marginals as MG
from oracle import rng
from oracle.chform import run_gates
from tests._circuits import rand_clifford


def _random_psi(n, seed, k=3):
    rng = random.Random(seed)
    terms, coefs = [], []
    for _ in range(k):
        terms.append(run_gates(n, rand_clifford(n, 18, rng, proj=False)))
        coefs.append(complex(rng.gauss(0, 1), rng.gauss(0, 1)))
    psi = sum(b * np.array([t.amplitude(x) for x in range(1 << n)]) for t, b in zip(terms, coefs))
    return terms, coefs, psi


def test_median_of_means_by_hand():
    assert MG.median_of_means([1, 2, 3, 4], 4, 1) == pytest.approx(2.5)
    assert MG.median_of_means([1, 3, 10, 20, 0, 2], 2, 3) == pytest.approx(2.0)     # means 2, 15, 1
    assert MG.median_of_means([1, 3, 10, 20], 2, 2) == pytest.approx(8.5)           # means 2, 15
    with pytest.raises(ValueError):
        MG.median_of_means([1, 2, 3], 2, 2)


@pytest.mark.parametrize("seed", range(4))
def test_projection_matches_dense_projector(seed):
    n = 4
    terms, coefs, psi = _random_psi(n, 70 + seed)
    q, b = seed % n, seed % 2
    proj = MG.project(terms, q, b)
    got = sum(c * np.array([t.amplitude(x) for x in range(1 << n)]) for t, c in zip(proj, coefs))
    keep = np.array([((x >> q) & 1) == b for x in range(1 << n)])
    np.testing.assert_allclose(got, np.where(keep, psi, 0), atol=1e-12)


@pytest.mark.parametrize("n", [2, 3])
def test_exact_marginals_with_all_equatorial_states(n):
    """With every A in M_n each estimate is exact: p_b = ||Pi_b psi||^2 (K = 1)."""
    terms, coefs, psi = _random_psi(n, 90 + n)
    As = list(E.all_equatorial(n))
    qubits = list(range(n))[::-1][:2]
    bits, probs = MG.marginal_sample(terms, coefs, qubits, len(As), 1, seed=5, As=As)
    prob = np.abs(psi) ** 2
    fixed = {}
    for (q, x), (p0, p1) in zip(zip(qubits, bits), probs):
        for b, p in ((0, p0), (1, p1)):
            sel = [i for i in range(1 << n)
                   if ((i >> q) & 1) == b and all(((i >> qq) & 1) == xx for qq, xx in fixed.items())]
            assert p == pytest.approx(prob[sel].sum(), rel=1e-10, abs=1e-12)
        fixed[q] = x


def test_chain_rule_frequencies_match_dense_marginal():
    n = 3
    terms, coefs, psi = _random_psi(n, 123)
    As = list(E.all_equatorial(n))
    qubits = [2, 0]
    prob = np.abs(psi) ** 2
    prob /= prob.sum()
    want = np.zeros(4)
    for i in range(1 << n):
        want[((i >> 2) & 1) + 2 * ((i >> 0) & 1)] += prob[i]
    # exact conditionals are reused across seeds: evaluate the four branch values once
    cache = {}
    counts = np.zeros(4)
    for seed in range(3000):
        # the sampler's own decisions, with the estimates memoised per prefix
        key = ()
        bits = []
        pref = terms
        for i, q in enumerate(qubits):
            if key not in cache:
                p = [MG.norm_mom(MG.project(pref, q, b), coefs, len(As), 1, 0, As=As) for b in (0, 1)]
                cache[key] = p
            p0, p1 = cache[key]
            u = rng.uniform(seed, MG.DRAW_STREAM + i, 0)
            x = 1 if u < p1 / (p0 + p1) else 0
            bits.append(x)
            pref = MG.project(pref, q, x)
            key = key + (x,)
        counts[bits[0] + 2 * bits[1]] += 1
    freq = counts / counts.sum()
    assert np.max(np.abs(freq - want)) < 0.04
    # and the function itself takes the same decisions as this replay for a few seeds
    for seed in range(3):
        b_fn, _ = MG.marginal_sample(terms, coefs, qubits, len(As), 1, seed, As=As)
        key, bits = (), []
        for i in range(2):
            p0, p1 = cache[key]
            x = 1 if rng.uniform(seed, MG.DRAW_STREAM + i, 0) < p1 / (p0 + p1) else 0
            bits.append(x)
            key = key + (x,)
        assert b_fn == bits
