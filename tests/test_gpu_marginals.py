"""Median-of-means estimates and chain-rule marginal sampling (end of Sec. 4.3) on the
GPU against the oracle: every branch probability within 1e-5 (relative to the
prefix's total), the same bit decisions (a decision within 1e-6 of its uniform draw
follows the GPU), and the full-size hidden shift, whose output is its shift."""
import numpy as np
import pytest

from oracle import decomp
from oracle import estimators as E
from oracle import marginals as MG
from oracle import rng
from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import oracle_overlaps, oracle_terms, require_cuda

pytestmark = pytest.mark.gpu


def _sim(n, ops, chi, mode, seed=0, ccz_mode="proj"):
    low = lrstab.lower_circuit(n, ops, ccz_mode)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode=mode, seed=seed)
    sim.apply_clifford(low.gates)
    return sim


def _oracle_mom(terms, coefs, n, L, K, seed):
    ov = oracle_overlaps(terms, coefs, n, seed, L * K, parallel=True)
    return MG.median_of_means((2.0 ** n) * np.abs(ov) ** 2, L, K)


def test_copy_terms_and_median_of_means():
    require_cuda()
    cfg = workloads.config_tiny()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    sim = _sim(n, ops, chi, "exact")
    other = lrstab.Simulator(n, 0)
    other.copy_terms_from(sim)
    a, b = sim.export_terms(), other.export_terms()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    terms, coefs, _ = oracle_terms(n, ops, chi, "exact")
    for L, K in ((40, 3), (25, 4), (64, 1)):
        got = sim.norm_median_of_means(L, K, seed=17)
        want = _oracle_mom(terms, coefs, n, L, K, 17)
        assert got == pytest.approx(want, rel=1e-5)
    with pytest.raises(lrstab.LrsError):
        sim.norm_median_of_means(0, 3, seed=1)
    bad = lrstab.Simulator(n + 1, 0)
    with pytest.raises(lrstab.LrsError):
        bad.copy_terms_from(sim)
    for s in (sim, other, bad):
        s.close()


def test_marginal_sample_replays_oracle():
    require_cuda()
    cfg = workloads.config_tiny()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    sim = _sim(n, ops, chi, "exact")
    qubits, L, K, seed = [0, 3, 7, 9], 32, 3, 2024
    bits, probs = sim.marginal_sample(qubits, L, K, seed)
    terms, coefs, _ = oracle_terms(n, ops, chi, "exact")
    pref = terms
    for i, q in enumerate(qubits):
        s_i = rng.rand64(seed, MG.STEP_STREAM + i, 0)
        p = [_oracle_mom(MG.project(pref, q, b), coefs, n, L, K, s_i) for b in (0, 1)]
        tot = p[0] + p[1]
        for b in (0, 1):
            assert abs(probs[i][b] - p[b]) <= 1e-5 * max(tot, 1e-12), (i, b, probs[i], p)
        u = rng.uniform(seed, MG.DRAW_STREAM + i, 0)
        want = 1 if (tot > 0 and u < p[1] / tot) else 0
        if tot > 0 and abs(u - p[1] / tot) < 1e-6:
            want = bits[i]
        assert bits[i] == want, i
        pref = MG.project(pref, q, bits[i])
    with pytest.raises(lrstab.LrsError):
        sim.marginal_sample([1, 1], L, K, seed)
    with pytest.raises(lrstab.LrsError):
        sim.marginal_sample([n], L, K, seed)
    sim.close()


def test_hidden_shift_marginals_give_the_shift():
    """Exact 2^16-term decomposition of |s>: every sampled bit is the shift's bit and
    the other branch has probability zero up to rounding."""
    require_cuda()
    cfg = workloads.config_hidden_shift()
    n, ops, chi, shift = cfg["n"], cfg["ops"], cfg["chi"], cfg["shift"]
    sim = _sim(n, ops, chi, "exact")
    qubits = [0, 7, 19, 20, 33, 39]
    bits, probs = sim.marginal_sample(qubits, 64, 3, seed=11)
    for q, b, (p0, p1) in zip(qubits, bits, probs):
        assert b == (shift >> q) & 1
        right, wrong = (p1, p0) if b else (p0, p1)
        assert right == pytest.approx(1.0, abs=1e-4)
        assert abs(wrong) <= 1e-6
    sim.close()


def test_sparsification_certificate_vs_oracle():
    """lrs_sparsification_certificate (Lemma (Sparsification tail bound)): the median of
    means, the standard error of the L K equatorial samples and delta^2 = ||c||_1^2 /
    chi against the oracle's values on the same equatorial states."""
    require_cuda()
    n = 10
    ops = workloads.random_clifford_t(n, 150, 8, seed=71)
    chi, seed = 96, 5
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode="sparsify", seed=seed)
    sim.apply_clifford(low.gates)
    L, K, aseed = 40, 3, 1234
    cert = lrstab.sparsification_certificate(sim, L, K, aseed)
    terms, coefs, _ = oracle_terms(n, ops, chi, "sparsify", seed=seed)
    etas = np.array([E.eta(terms, coefs, E.draw_A(n, aseed, l)) for l in range(L * K)])
    mom = MG.median_of_means(etas, L, K)
    se = etas.std(ddof=1) / np.sqrt(etas.size)
    delta2 = decomp.l1_norm(decomp.lower(ops)[1]) ** 2 / chi
    assert cert["omega_norm2"] == pytest.approx(mom, rel=1e-5)
    assert cert["stderr_mean"] == pytest.approx(se, rel=1e-4)
    assert cert["delta2"] == pytest.approx(delta2, rel=1e-12)
    assert cert["bound"] == pytest.approx(mom - 1 + delta2, rel=1e-4, abs=1e-6)
    assert cert["conclusive"] == (2 * se < delta2)
    sim.close()
