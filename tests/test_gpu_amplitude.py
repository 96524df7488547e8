"""Amplitude parity: CUDA <x|psi> against the FP64 oracle (and the dense state
vector where n is small).  Tolerance: |a_gpu - a| <= 1e-5 max(|a|, ||psi|| 2^{-n/2})."""
import math

import numpy as np
import pytest
import torch

from oracle import dense, exact
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


def _amps_err(sim, xs):
    x = torch.tensor(np.asarray(xs, dtype=np.uint64).view(np.int64), device="cuda:0")
    err = torch.empty(len(xs), dtype=torch.float32, device="cuda:0")
    out = sim.amplitude(x, err=err).cpu().numpy()
    return out[:, 0] + 1j * out[:, 1], err.cpu().numpy().astype(np.float64)


def _check_vs_oracles(got, err, terms, coefs, chs, ex, xs, n, norm):
    """FP64 oracle within the 1e-5 tolerance; exact Z[zeta8] sum within the kernel's
    stated per-result bound.  Returns the measured errors against the exact sums."""
    want = np.array([E.amplitude(terms, coefs, x) for x in xs])
    exc = np.array([exact.to_complex(ex.amplitude(terms, chs, x)) for x in xs])
    assert np.all(np.abs(got - want) <= amp_tol(want, n, norm))
    d = np.abs(got - exc)
    assert np.all(d <= err), f"bound violated: max d/err = {np.max(d / np.maximum(err, 1e-300)):.3g}"
    # the FP64 oracle is itself within 1e-12 of the exact sum
    assert np.all(np.abs(want - exc) <= 1e-12 * np.maximum(np.abs(exc), norm * 2.0 ** (-n / 2)))
    return d


@pytest.mark.parametrize("n", [50, 56, 63, 64])
def test_wide_registers_vs_oracle_and_exact(n):
    """n = 50..64: Four-Russians tables of 13..16 chunks, packed (n <= 62) and the
    unpacked form n > 62, against the FP64 oracle and the exact chi-sums; 300 ragged
    terms of a sparsified Clifford+T circuit, strings drawn from the terms plus random
    ones."""
    require_cuda()
    ops = workloads.random_clifford_t(n, 160, 8, seed=500 + n)
    chi, seed = 300, 17
    sim = _sim(n, ops, chi, "sparsify", seed=seed)
    terms, coefs, chs = oracle_terms(n, ops, chi, "sparsify", seed=seed, parallel=True)
    ex = exact.ExactDecomposition(n, ops, chi, "sparsify")
    xs = [terms[i].sample(0x9E3779B9 * (i + 3)) for i in range(0, chi, 3)]
    xs += [int(x) for x in workloads.random_bitstrings(n, 28, seed=n)]
    got, err = _amps_err(sim, xs)
    norm = abs(coefs[0]) * np.sqrt(chi)          # incoherent scale of the terms
    _check_vs_oracles(got, err, terms, coefs, chs, ex, xs, n, norm)
    assert np.count_nonzero(np.abs(got) > 0) >= len(xs) // 2
    sim.close()


@pytest.mark.parametrize("beta", [0.2, math.pi / 4], ids=["beta_0.2", "beta_pi_4"])
def test_qaoa_n50_slice_vs_oracle_and_exact(beta):
    """The QAOA Max-E3LIN2 workload at n = 50 (gamma 0.3, beta 0.2, 116 rotation
    slots; chi = 2^20 sparsified terms) and the paper's line beta = pi/4 (its 50 mixer
    slots are Clifford, one choice each): a 256-term slice of that decomposition,
    strings sampled from the slice's terms plus random ones, against the FP64 oracle
    and the exact chi-sums, with the per-result bound checked."""
    require_cuda()
    cfg = workloads.config_qaoa(beta=beta)
    n, ops, chi_total, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    alpha0, chi = 777_777, 256
    sim = _sim(n, ops, chi, "sparsify", seed=seed, alpha0=alpha0, chi_total=chi_total)
    terms, coefs, chs = oracle_terms(n, ops, chi_total, "sparsify", seed=seed,
                                     alphas=range(alpha0, alpha0 + chi), parallel=True)
    ex = exact.ExactDecomposition(n, ops, chi_total, "sparsify")
    xs = [terms[i].sample(0x5DEECE66D * (i + 1)) for i in range(0, chi, 2)]
    xs += [int(x) for x in workloads.random_bitstrings(n, 64, seed=4)]
    got, err = _amps_err(sim, xs)
    norm = abs(coefs[0]) * np.sqrt(chi)
    d = _check_vs_oracles(got, err, terms, coefs, chs, ex, xs, n, norm)
    scale = np.maximum(np.abs(got), norm * 2.0 ** (-n / 2))
    assert np.max(d / scale) < 1e-6
    assert np.count_nonzero(np.abs(got) > 0) >= 100
    sim.close()


def test_error_bound_full_size_mid():
    """At the full n = 40, 2^16-term size the stated bound is finite, positive where
    terms contribute, and small against the 1e-5 tolerance (||psi|| ~ 1)."""
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, chi, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    sim = _sim(n, ops, chi, "sparsify", seed=seed)
    xs = sim.sample_terms(1024, seed=31).cpu().numpy().view(np.uint64)
    got, err = _amps_err(sim, xs)
    assert np.all(np.isfinite(err)) and np.all(err > 0)
    assert np.max(err) < 1e-5 * 2.0 ** (-n / 2)
    # the bound and the plain call agree on the values
    plain = _amps(sim, xs)
    assert np.array_equal(plain, got)
    sim.close()
