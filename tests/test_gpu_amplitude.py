"""Amplitude parity: CUDA <x|psi> against the FP64 oracle (and the dense state
vector where n is small).  Tolerance: |a_gpu - a| <= 1e-5 max(|a|, ||psi|| 2^{-n/2})."""
import numpy as np
import pytest
import torch

from oracle import dense
from oracle import estimators as E
from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import amp_tol, oracle_terms, require_cuda

pytestmark = pytest.mark.gpu


def _sim(n, ops, chi, mode, seed=0, ccz_mode="proj", alpha0=0, chi_total=None):
    low = lrstab.lower_circuit(n, ops, ccz_mode)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode=mode, seed=seed, alpha0=alpha0, chi_total=chi_total)
    sim.apply_clifford(low.gates)
    return sim


def _amps(sim, xs):
    x = torch.tensor(np.asarray(xs, dtype=np.uint64).view(np.int64), device="cuda:0")
    out = sim.amplitude(x).cpu().numpy()
    return out[:, 0] + 1j * out[:, 1]


def test_tiny_all_amplitudes_vs_oracle_and_dense():
    require_cuda()
    cfg = workloads.config_tiny()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    sim = _sim(n, ops, chi, "exact")
    got = _amps(sim, np.arange(1 << n))
    terms, coefs, _ = oracle_terms(n, ops, chi, "exact")
    want = np.array([E.amplitude(terms, coefs, x) for x in range(1 << n)])
    psi = dense.run(n, ops)
    np.testing.assert_allclose(want, psi, atol=1e-12)
    assert np.all(np.abs(got - want) <= amp_tol(want, n))
    assert abs(np.sum(np.abs(got) ** 2) - 1.0) < 1e-5
    sim.close()


def test_ragged_tiles_and_batch():
    """chi = 600 (four full 128-term tiles and a tail), batch = 100 (ragged)."""
    require_cuda()
    n = 12
    ops = workloads.random_clifford_t(n, 200, 9, seed=44)
    chi = 600
    sim = _sim(n, ops, chi, "sparsify", seed=5)
    xs = workloads.random_bitstrings(n, 100, seed=8)
    got = _amps(sim, xs)
    terms, coefs, _ = oracle_terms(n, ops, chi, "sparsify", seed=5, parallel=True)
    want = np.array([E.amplitude(terms, coefs, int(x)) for x in xs])
    norm = np.sqrt(np.sum(np.abs([E.amplitude(terms, coefs, x) for x in range(1 << n)]) ** 2))
    assert np.all(np.abs(got - want) <= amp_tol(want, n, norm))
    sim.close()


def test_empty_batch_and_bad_args():
    require_cuda()
    sim = _sim(4, [("H", 0), ("T", 0)], 2, "exact")
    x = torch.empty(0, dtype=torch.int64, device="cuda:0")
    out = sim.amplitude(x)
    assert out.shape == (0, 2)
    with pytest.raises(lrstab.LrsError):
        sim.apply_clifford(lrstab.gates_array([("CX", 1, 1)]))
    with pytest.raises(lrstab.LrsError):
        sim.apply_clifford(lrstab.gates_array([("H", 4)]))
    with pytest.raises(lrstab.LrsError):
        sim.norm_estimate(0, seed=1)
    sim.close()


def test_mid_slice_vs_oracle():
    """n=40, 2000 Cliffords + 24 T: a 256-term slice of the 2^16-term decomposition."""
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, chi_total, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    alpha0, chi = 4000, 256
    sim = _sim(n, ops, chi, "sparsify", seed=seed, alpha0=alpha0, chi_total=chi_total)
    terms, coefs, _ = oracle_terms(n, ops, chi_total, "sparsify", seed=seed,
                                   alphas=range(alpha0, alpha0 + chi), parallel=True)
    # x drawn from the slice's own terms (so amplitudes are not all zero) plus random x
    xs = [terms[i].sample(0x5DEECE66D * (i + 1)) for i in range(0, chi, 8)]
    xs += [int(x) for x in workloads.random_bitstrings(n, 16, seed=3)]
    got = _amps(sim, xs)
    want = np.array([E.amplitude(terms, coefs, x) for x in xs])
    # ||psi|| of the full decomposition is ~1; a 256-term slice carries weight ~ sqrt(256/2^16)
    norm = np.sqrt(chi / chi_total)
    assert np.all(np.abs(got - want) <= amp_tol(want, n, norm))
    assert np.count_nonzero(np.abs(want) > 0) >= len(xs) // 2
    sim.close()


def test_mid_full_size_equals_sum_of_shards():
    """Full 2^16-term launch (the benchmark's configuration) against four
    2^14-term shards: the amplitude is linear in the terms."""
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, chi, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    xs = workloads.random_bitstrings(n, 512, seed=11)
    full = _sim(n, ops, chi, "sparsify", seed=seed)
    # add strings sampled from the terms so that many amplitudes are nonzero
    xt = full.sample_terms(512, seed=12).cpu().numpy().view(np.uint64)
    allx = np.concatenate([xs, xt])
    a_full = _amps(full, allx)
    full.close()
    acc = np.zeros(len(allx), complex)
    for k in range(4):
        sh = _sim(n, ops, chi // 4, "sparsify", seed=seed, alpha0=k * chi // 4, chi_total=chi)
        acc += _amps(sh, allx)
        sh.close()
    assert np.all(np.abs(a_full - acc) <= amp_tol(acc, n, 1.0))
    assert np.count_nonzero(np.abs(acc) > 1e-3 * 2 ** (-n / 2)) > 256


def test_hidden_shift_full_size_outputs_shift():
    """Exact 2^16-term decomposition of the 40-qubit hidden-shift circuit:
    <s|psi> = 1 and <x|psi> = 0 for x != s (Sec. 2.4.2)."""
    require_cuda()
    cfg = workloads.config_hidden_shift()
    n, ops, chi, s = cfg["n"], cfg["ops"], cfg["chi"], cfg["shift"]
    sim = _sim(n, ops, chi, "exact")
    xs = [s] + [s ^ (1 << j) for j in range(n)] + [int(x) for x in workloads.random_bitstrings(n, 64, 5)]
    got = _amps(sim, xs)
    assert abs(got[0] - 1.0) <= 1e-5
    assert np.all(np.abs(got[1:]) <= 1e-5 * 2 ** (-n / 2))
    sim.close()
