"""Pins for the oracle CH-form simulator (Sec. 4.1) against dense brute force."""
import random

import numpy as np
import pytest

from oracle import dense
from oracle.chform import CHForm, bit, popcount, run_gates, single_qubit_form
from tests._circuits import rand_clifford


def _all_amps(ch, n):
    return np.array([ch.amplitude(x) for x in range(1 << n)])


@pytest.mark.parametrize("proj", [False, True])
def test_chform_matches_dense(proj):
    """Every amplitude of random Clifford (+projector) circuits equals the dense vector."""
    rng = random.Random(11 + proj)
    for _ in range(250):
        n = rng.randrange(1, 8)
        ops = rand_clifford(n, rng.randrange(1, 45), rng, proj=proj)
        ch = run_gates(n, ops)
        psi = dense.run(n, ops)
        np.testing.assert_allclose(_all_amps(ch, n), psi, atol=1e-12)


def test_each_gate_against_dense_after_every_step():
    """Parity after every single gate catches an error in any one rule."""
    rng = random.Random(3)
    for _ in range(40):
        n = rng.randrange(2, 7)
        ops = rand_clifford(n, 30, rng, proj=True)
        ch = CHForm(n)
        psi = dense.zero_state(n)
        for g in ops:
            run_gates(n, [g], ch)
            psi = dense.apply_gate(psi, n, g)
            np.testing.assert_allclose(_all_amps(ch, n), psi, atol=1e-12, err_msg=str(g))


def test_tableau_invariants():
    """F G^T = I (mod 2) and M F^T symmetric (mod 2) after every gate (Sec. 4.1, 4.3)."""
    rng = random.Random(5)
    for _ in range(60):
        n = rng.randrange(1, 9)
        ch = CHForm(n)
        for g in rand_clifford(n, 40, rng, proj=True):
            run_gates(n, [g], ch)
            for a in range(n):
                for b in range(n):
                    fg = popcount(ch.F[a] & ch.G[b]) & 1
                    assert fg == (1 if a == b else 0)
                    mf_ab = popcount(ch.M[a] & ch.F[b]) & 1
                    mf_ba = popcount(ch.M[b] & ch.F[a]) & 1
                    assert mf_ab == mf_ba


def test_unit_norm_of_unitary_terms():
    """sum_x |<x|phi>|^2 = 1 for every stabilizer state reached by unitary gates."""
    rng = random.Random(9)
    for _ in range(80):
        n = rng.randrange(1, 9)
        ch = run_gates(n, rand_clifford(n, 50, rng))
        assert abs(np.sum(np.abs(_all_amps(ch, n)) ** 2) - 1) < 1e-12
        assert ch.h == 0 and not ch.zero


def test_hadamard_on_zero_state():
    """H_p|0^n> gives V_0 = {p}, V_C = I, (a,b,c) = (0,1,0): v = e_p, s = 0, omega = 1."""
    for n in (1, 5, 64):
        for p in (0, n - 1):
            ch = CHForm(n)
            ch.apply_H(p)
            assert ch.v == 1 << p and ch.s == 0 and ch.k % 8 == 0 and ch.h == 0
            assert ch.F == [1 << j for j in range(n)] and ch.M == [0] * n


def test_single_qubit_rewrite_table():
    """The brute-force rewrite agrees with the explicit 2-vector for all 16 inputs."""
    r2 = 1 / np.sqrt(2)
    Hm = np.array([[r2, r2], [r2, -r2]])
    Sm = np.diag([1, 1j])
    for vq in (0, 1):
        for yq in (0, 1):
            for d in range(4):
                zq = 1 - yq
                vec = np.zeros(2, complex)
                vec[yq] += 1
                vec[zq] += 1j ** d
                if vq:
                    vec = Hm @ vec
                a, b, c, k = single_qubit_form(vq, yq, zq, d)
                e = np.zeros(2, complex)
                e[c] = 1
                got = np.sqrt(2) * np.exp(1j * np.pi * k / 4) * (
                    np.linalg.matrix_power(Sm, a) @ np.linalg.matrix_power(Hm, b) @ e)
                np.testing.assert_allclose(got, vec, atol=1e-12)
                if b == 0:
                    assert a == 0


def test_sampling_support_and_uniformity():
    """x = w G^T with w_j = s_j on v_j = 0 reaches exactly the support, uniformly."""
    rng = random.Random(21)
    for _ in range(30):
        n = rng.randrange(1, 7)
        ch = run_gates(n, rand_clifford(n, 30, rng))
        amps = _all_amps(ch, n)
        support = {x for x in range(1 << n) if abs(amps[x]) > 1e-9}
        seen = {}
        for flips in range(1 << n):
            if flips & ~ch.v:
                continue
            x = ch.sample(flips)
            seen[x] = seen.get(x, 0) + 1
        assert set(seen) == support
        assert len(set(seen.values())) == 1
        assert len(support) == 1 << popcount(ch.v)


@pytest.mark.parametrize("n", [10, 11, 12])
def test_chform_matches_dense_up_to_12_qubits(n):
    """The same brute-force pin at n = 10..12 (all 2^n amplitudes), with a check after
    every gate on one circuit at n = 10."""
    rng = random.Random(100 + n)
    for trial in range(3):
        ops = rand_clifford(n, 80, rng, proj=False)
        q = rng.randrange(n)
        # a projector that keeps part of the state (one of P0, P1 always does)
        proj = "P0" if np.abs(dense.run(n, ops + [("P0", q)])).max() > 0 else "P1"
        ops += [(proj, q), ("H", rng.randrange(n))]
        ch = run_gates(n, ops)
        psi = dense.run(n, ops)
        assert np.abs(psi).max() > 0
        np.testing.assert_allclose(_all_amps(ch, n), psi, atol=1e-12)
    if n == 10:
        ch = CHForm(n)
        psi = dense.zero_state(n)
        for g in rand_clifford(n, 40, rng, proj=True):
            run_gates(n, [g], ch)
            psi = dense.apply_gate(psi, n, g)
            np.testing.assert_allclose(_all_amps(ch, n), psi, atol=1e-12, err_msg=str(g))
