"""Pins for the oracle's norm estimation (Sec. 4.3) and Metropolis chain (Sec. 4.2)."""
import random

import numpy as np
import pytest

from oracle import decomp, dense
from oracle import estimators as E
from oracle.chform import run_gates
from paper_1808_00128_gb300 import workloads
from tests._circuits import rand_clifford


def test_inner_product_matches_dense():
    rng = random.Random(31)
    for trial in range(150):
        n = rng.randrange(1, 7)
        ops = rand_clifford(n, rng.randrange(1, 35), rng, proj=trial % 3 == 0)
        ch = run_gates(n, ops)
        if ch.zero:
            continue
        A = E.draw_A(n, 5, trial)
        want = np.vdot(dense.run(n, ops), dense.equatorial_state(n, A))   # <phi|phi_A>
        got = np.conj(ch.omega()) * E.inner_equatorial(ch, A)
        assert abs(got - want) < 1e-12


def test_draw_A_is_in_Mn():
    for n in (1, 5, 40, 64):
        A = E.draw_A(n, 3, 7)
        assert (A == A.T).all()
        assert set(np.diag(A)) <= {0, 1, 2, 3}
        off = A[~np.eye(n, dtype=bool)]
        assert set(off) <= {0, 1}


@pytest.mark.parametrize("n", [1, 2, 3])
def test_exhaustive_average_equals_norm(n):
    """E_A eta_A = ||psi||^2 exactly and Var <= ||psi||^4 (Lemma (Norm Estimation)),
    averaging over all of M_n for a random unnormalised superposition."""
    rng = random.Random(40 + n)
    terms, coefs = [], []
    for _ in range(3):
        terms.append(run_gates(n, rand_clifford(n, 15, rng, proj=True)))
        coefs.append(complex(rng.gauss(0, 1), rng.gauss(0, 1)))
    psi = sum(b * np.array([t.amplitude(x) for x in range(1 << n)]) for t, b in zip(terms, coefs))
    norm2 = np.linalg.norm(psi) ** 2
    etas = np.array([E.eta(terms, coefs, A) for A in E.all_equatorial(n)])
    assert etas.mean() == pytest.approx(norm2, rel=1e-12)
    assert etas.var() <= norm2 ** 2 * (1 + 1e-12)


def test_norm_estimate_unit_for_exact_decomposition():
    ops = workloads.random_clifford_t(8, 80, 4, seed=3)
    terms, coefs, _ = decomp.build_decomposition(8, ops, chi=16, mode="exact")
    _, mean = E.norm_estimate(terms, coefs, L=200, seed=1)
    assert mean == pytest.approx(1.0, abs=0.25)


def test_metropolis_rule_has_P_stationary():
    """The single-flip Metropolis kernel T(x->y) of Sec. 4.2 satisfies P T = P."""
    n = 4
    ops = workloads.random_clifford_t(n, 40, 3, seed=8)
    psi = dense.run(n, ops)
    P = np.abs(psi) ** 2
    T = np.zeros((16, 16))
    for x in range(16):
        for j in range(n):
            y = x ^ (1 << j)
            if P[x] == 0:
                acc = 1.0
            else:
                acc = 1.0 if P[y] >= P[x] else P[y] / P[x]
            T[x, y] += acc / n
            T[x, x] += (1 - acc) / n
    np.testing.assert_allclose(P @ T, P, atol=1e-14)


def test_metropolis_draws_in_range():
    for c in range(20):
        for t in range(50):
            j, r = E.metropolis_draws(50, 7, c, t)
            assert 0 <= j < 50 and 0.0 <= r < 1.0


def test_metropolis_chain_matches_distribution():
    """Long oracle chains on a small exact decomposition reproduce |<x|psi>|^2."""
    n = 4
    ops = [("H", 0), ("H", 1), ("H", 2), ("H", 3), ("T", 0), ("CX", 0, 1), ("T", 1),
           ("H", 1), ("CZ", 1, 2), ("T", 2), ("H", 2), ("CX", 2, 3)]
    terms, coefs, _ = decomp.build_decomposition(n, ops, chi=8, mode="exact")
    P = np.array([E.probability(terms, coefs, x) for x in range(16)])
    P /= P.sum()
    counts = np.zeros(16)
    x = int(np.argmax(P))
    px = E.probability(terms, coefs, x)
    for t in range(20000):
        x, px, *_ = E.metropolis_step(terms, coefs, x, px, n, seed=4, chain=0, step=t)
        counts[x] += 1
    emp = counts / counts.sum()
    assert 0.5 * np.abs(emp - P).sum() < 0.05


def test_hidden_shift_outputs_shift():
    """The hidden-shift circuit maps |0^n> to |s> (Sec. 2.4.2), dense and decomposed."""
    ops, s = workloads.hidden_shift_circuit(8, 4, seed=12)
    psi = dense.run(8, ops)
    assert abs(psi[s]) == pytest.approx(1.0, abs=1e-12)
    terms, coefs, _ = decomp.build_decomposition(8, ops, chi=16, mode="exact", ccz_mode="proj")
    assert E.amplitude(terms, coefs, s) == pytest.approx(psi[s], abs=1e-12)
    for x in (0, s ^ 1, s ^ 0x80, 0x55):
        assert abs(E.amplitude(terms, coefs, x)) < 1e-12
