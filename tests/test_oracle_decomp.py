"""Pins for the oracle's sum-over-Cliffords decompositions (Sec. 2.3.2, Sec. 5.2)."""
import math
import random

import numpy as np
import pytest

from oracle import decomp, dense
from oracle.estimators import amplitude
from paper_1808_00128_gb300 import workloads


def _lin_comb_matrix(n, dec):
    return sum(c * dense.gate_matrix(n, gates) for c, gates in dec)


@pytest.mark.parametrize("op", [("T", 0), ("RZ", 0, 0.3), ("RZ", 0, -0.3), ("RZ", 0, 0.4),
                                ("RZ", 0, math.pi / 2), ("RZ", 0, -1.1)])
def test_rotation_decomposition_is_exact(op):
    dec = decomp.gate_decomposition(op)
    np.testing.assert_allclose(_lin_comb_matrix(1, dec), dense.gate_matrix(1, [op]), atol=1e-14)


@pytest.mark.parametrize("kind", ["CCZ_SUM8", "CCZ_PROJ"])
def test_ccz_decomposition_is_exact(kind):
    dec = decomp.gate_decomposition((kind, 0, 1, 2))
    np.testing.assert_allclose(_lin_comb_matrix(3, dec), dense.gate_matrix(3, [("CCZ", 0, 1, 2)]),
                               atol=1e-14)


def test_l1_norms_match_stabilizer_extent():
    """||c||_1^2 equals xi for the optimal decompositions (Sec. 2.3.2, 2.4.2)."""
    t = decomp.gate_decomposition(("T", 0))
    xi_t = sum(abs(c) for c, _ in t) ** 2
    assert xi_t == pytest.approx(1 / math.cos(math.pi / 8) ** 2, rel=1e-14)   # 1/F(T)
    for th in (0.1, 0.3, 0.4, 1.2):
        r = decomp.gate_decomposition(("RZ", 0, th))
        xi = sum(abs(c) for c, _ in r) ** 2
        want = (math.cos(th / 2) + math.tan(math.pi / 8) * math.sin(th / 2)) ** 2
        assert xi == pytest.approx(want, rel=1e-13)
    ccz = decomp.gate_decomposition(("CCZ_SUM8", 0, 1, 2))
    assert sum(abs(c) for c, _ in ccz) ** 2 == pytest.approx(16 / 9, rel=1e-14)


def test_exact_decomposition_reproduces_circuit():
    ops = workloads.random_clifford_t(6, 60, 4, seed=5)
    terms, coefs, _ = decomp.build_decomposition(6, ops, chi=16, mode="exact")
    psi = dense.run(6, ops)
    amps = np.array([amplitude(terms, coefs, x) for x in range(64)])
    np.testing.assert_allclose(amps, psi, atol=1e-12)


def test_exact_ccz_projector_decomposition():
    ops = [("H", 0), ("H", 1), ("H", 2), ("H", 3), ("CCZ", 0, 1, 3), ("H", 3), ("CX", 3, 2),
           ("CCZ", 1, 2, 3), ("H", 1)]
    terms, coefs, _ = decomp.build_decomposition(4, ops, chi=4, mode="exact", ccz_mode="proj")
    psi = dense.run(4, ops)
    amps = np.array([amplitude(terms, coefs, x) for x in range(16)])
    np.testing.assert_allclose(amps, psi, atol=1e-12)


def test_sparsification_expected_error():
    """E||psi - Omega||^2 = (||c||_1^2 - ||psi||^2) / k, computed exactly over the
    choice distribution (proof of Lemma (Sparsification)); this is at most the
    lemma's ||c||_1^2 / k."""
    n = 3
    ops = [("H", 0), ("T", 0), ("H", 1), ("CX", 0, 1), ("T", 1), ("H", 2), ("RZ", 2, 0.3),
           ("CZ", 1, 2), ("H", 0)]
    gates, slots = decomp.lower(ops)
    psi = dense.run(n, ops)
    l1 = decomp.l1_norm(slots)
    # single-draw state omega (k = 1): ||c||_1 * prod phase * phi_choices
    exp_err = 0.0
    exp_state = np.zeros(1 << n, complex)
    for choice in np.ndindex(*[len(d) for d in slots]):
        p = np.prod([abs(slots[s][j][0]) / sum(abs(c) for c, _ in slots[s])
                     for s, j in enumerate(choice)])
        ch = decomp.build_term(n, gates, slots, list(choice))
        b = decomp.coefficient(slots, list(choice), "sparsify", chi=1)
        om = b * np.array([ch.amplitude(x) for x in range(1 << n)])
        exp_err += p * np.linalg.norm(psi - om) ** 2
        exp_state += p * om
    np.testing.assert_allclose(exp_state, psi, atol=1e-12)      # E[Omega] = psi
    assert exp_err == pytest.approx(l1 ** 2 - 1.0, rel=1e-12)   # k = 1
    assert exp_err <= l1 ** 2


def test_sparsify_choice_frequencies():
    dec = decomp.gate_decomposition(("RZ", 0, 0.3))
    p1 = abs(dec[1][0]) / sum(abs(c) for c, _ in dec)
    us = (np.arange(100000) + 0.5) / 100000
    freq = np.mean([decomp.choice_sparsify(dec, u) == 1 for u in us])
    assert freq == pytest.approx(p1, abs=2e-5)


def test_sparsified_norm_concentrates():
    """<Omega|Omega> -> ||psi||^2 = 1 as k grows (Lemma (Sparsification tail bound))."""
    n = 4
    ops = workloads.random_clifford_t(n, 30, 3, seed=2)
    psi = dense.run(n, ops)
    terms, coefs, _ = decomp.build_decomposition(n, ops, chi=2000, mode="sparsify", seed=99)
    amps = np.array([amplitude(terms, coefs, x) for x in range(1 << n)])
    assert np.linalg.norm(amps) ** 2 == pytest.approx(1.0, abs=0.05)
    assert np.linalg.norm(amps - psi) ** 2 < 3 * (decomp.l1_norm(decomp.lower(ops)[1]) ** 2) / 2000


@pytest.mark.parametrize("seed", range(6))
def test_gadget_form_equals_circuit_state(seed):
    """Fixed-sample gadgets (Eq. (Uidentity)): the exact decomposition on n + tau
    qubits is U|0^n> (x) |0^tau> (ancillas in the high bits), for T, RZ and CCZ in
    both CCZ forms."""
    rng = random.Random(600 + seed)
    n = rng.randint(3, 4)
    ops = []
    for _ in range(12):
        r = rng.random()
        if r < 0.3:
            ops.append(("H", rng.randrange(n)))
        elif r < 0.5:
            a, b = rng.sample(range(n), 2)
            ops.append(("CX", a, b))
        elif r < 0.6:
            ops.append(("S", rng.randrange(n)))
        elif r < 0.7:
            a, b = rng.sample(range(n), 2)
            ops.append(("CZ", a, b))
    pos = rng.sample(range(len(ops) + 1), 3)
    extra = [("T", rng.randrange(n)), ("RZ", rng.randrange(n), rng.uniform(-2.0, 2.0)),
             ("CCZ",) + tuple(rng.sample(range(n), 3))]
    for p_, e in sorted(zip(pos, extra), reverse=True):
        ops.insert(p_, e)
    want = dense.run(n, ops)
    for ccz_mode in ("proj", "sum8"):
        n_total, gates, slots = decomp.lower_gadget(n, ops, ccz_mode)
        assert n_total == n + 1 + 1 + 3
        chi = decomp.exact_chi(slots)
        terms, coefs, _ = decomp.build_decomposition(n, ops, chi, "exact", ccz_mode=ccz_mode, method="gadget")
        psi = sum(b * np.array([t.amplitude(x) for x in range(1 << n_total)]) for t, b in zip(terms, coefs))
        np.testing.assert_allclose(psi[: 1 << n], want, atol=1e-10)
        assert np.abs(psi[1 << n:]).max() < 1e-10
