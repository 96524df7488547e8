"""Fixed-sample gadget form (Sec. 2.3.1, Eq. (Uidentity)) on the GPU: tableaux
bit-exact against the oracle's gadget decomposition, amplitudes of the n + tau-qubit
state equal to those of the sum-over-Cliffords decomposition of the same circuit
(both exact), ancilla bits post-selected to zero, and a hidden shift with gadgets
outputting its shift."""
import numpy as np
import pytest
import torch

from oracle import decomp
from oracle import estimators as E
from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import compare_term, require_cuda

pytestmark = pytest.mark.gpu


def _sim(n, ops, method, ccz_mode="proj"):
    low = lrstab.lower_circuit(n, ops, ccz_mode, method=method)
    chi = low.exact_chi
    sim = lrstab.Simulator(low.n_total, 0)
    sim.init_terms(low, chi, mode="exact")
    sim.apply_clifford(low.gates)
    return sim, low, chi


def _amps(sim, xs):
    a = sim.amplitude(torch.from_numpy(np.asarray(xs, np.uint64).view(np.int64)).cuda()).cpu().numpy()
    return a[:, 0] + 1j * a[:, 1]


def test_tiny_gadget_terms_and_amplitudes():
    require_cuda()
    cfg = workloads.config_tiny()
    n, ops = cfg["n"], cfg["ops"]
    g, low, chi = _sim(n, ops, "gadget")
    assert low.n_total == n + 6 and chi == 64
    terms, coefs, _ = decomp.build_decomposition(n, ops, chi, "exact", method="gadget")
    ex = g.export_terms()
    for i, t in enumerate(terms):
        compare_term(ex, i, t, f"gadget term {i}")
    s, _, _ = _sim(n, ops, "sum")
    xs = np.arange(1 << n, dtype=np.uint64)
    ag, asum = _amps(g, xs), _amps(s, xs)
    np.testing.assert_allclose(ag, asum, atol=1e-5)
    want = np.array([E.amplitude(terms, coefs, int(x)) for x in xs[:64]])
    np.testing.assert_allclose(ag[:64], want, atol=1e-5)
    # any ancilla bit set: amplitude zero (post-selected)
    xa = xs[:128] | (np.uint64(1) << np.uint64(n + 2))
    assert np.abs(_amps(g, xa)).max() <= 1e-6
    g.close()
    s.close()


def test_gadget_matches_sum_over_cliffords_at_n30():
    """n=30, 14 T gates: gadget form on 44 qubits vs sum-over-Cliffords on 30, 2^14
    exact terms each, 512 strings."""
    require_cuda()
    n = 30
    ops = workloads.random_clifford_t(n, 600, 14, seed=workloads.SEED_BASE + 61)
    g, low, chi = _sim(n, ops, "gadget")
    assert low.n_total == n + 14 and chi == 1 << 14
    s, _, chi_s = _sim(n, ops, "sum")
    assert chi_s == chi
    xs = np.concatenate([workloads.random_bitstrings(n, 256, 7),
                         s.sample_terms(256, seed=3).cpu().numpy().view(np.uint64)])
    ag, asum = _amps(g, xs), _amps(s, xs)
    scale = max(np.abs(asum).max(), 2.0 ** (-n / 2))
    assert np.abs(ag - asum).max() <= 1e-5 * scale
    g.close()
    s.close()


def test_hidden_shift_with_gadgets_outputs_shift():
    require_cuda()
    ops, shift = workloads.hidden_shift_circuit(20, 4, workloads.SEED_BASE + 62)
    g, low, chi = _sim(20, ops, "gadget")
    assert low.n_total == 32
    a = _amps(g, [shift, shift ^ 1, shift ^ (1 << 7)])
    assert abs(a[0] - 1) <= 1e-5 and abs(a[1]) <= 1e-6 and abs(a[2]) <= 1e-6
    g.close()
