"""Norm-estimation parity: CUDA eta_l = 2^n |<phi_{A_l}|psi>|^2 against the oracle
(Lemmas (Inner Product), (Exponential Sum)) on the same A_l.  Tolerance
|eta_gpu - eta| <= 1e-5 max(eta, ||psi||^2)."""
import random

import numpy as np
import pytest

from oracle import estimators as E
from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import oracle_overlaps, oracle_terms, require_cuda

pytestmark = pytest.mark.gpu


def _sim(n, ops, chi, mode, seed=0, ccz_mode="proj", alpha0=0, chi_total=None):
    low = lrstab.lower_circuit(n, ops, ccz_mode)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode=mode, seed=seed, alpha0=alpha0, chi_total=chi_total)
    sim.apply_clifford(low.gates)
    return sim


# per-term paths of the kernel: -1 forms K = G^T (A+J) G for every term; 0 sums over
# y = G x for terms with v = all qubits; 12 for terms with up to 12 qubits outside v,
# their constraints folded while the rows are formed (up to 8) or one pass each
# ("seq": every constraint in its own pass)
FOLDS = (-1, 0, 12, "seq")


def _etas(sim, L, seed):
    out = {}
    for f in FOLDS:
        sim.set_tuning("norm_max_folds", 12 if f == "seq" else f)
        sim.set_tuning("norm_fuse_folds", 0 if f == "seq" else 8)
        out[f] = sim.norm_estimate(L, seed=seed).cpu().numpy()
    sim.set_tuning("norm_max_folds", 12)
    sim.set_tuning("norm_fuse_folds", 8)
    return out


def _check(eta_gpu, overl, n, norm2):
    if isinstance(eta_gpu, dict):
        for f, e in eta_gpu.items():
            _check(e, overl, n, norm2)
        return
    want = (2.0 ** n) * np.abs(overl) ** 2
    tol = 1e-5 * np.maximum(want, norm2)
    bad = np.abs(eta_gpu - want) > tol
    assert not bad.any(), (np.flatnonzero(bad)[:5], eta_gpu[bad][:5], want[bad][:5])


def test_tiny_config_eta_parity():
    require_cuda()
    cfg = workloads.config_tiny()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    sim = _sim(n, ops, chi, "exact")
    L = 96                                       # one full block of 64 A's and a tail
    eta, mean = sim.norm_estimate(L, seed=21, want_mean=True)
    terms, coefs, _ = oracle_terms(n, ops, chi, "exact")
    ov = oracle_overlaps(terms, coefs, n, 21, L, parallel=True)
    _check(eta.cpu().numpy(), ov, n, 1.0)
    _check(_etas(sim, L, 21), ov, n, 1.0)
    assert mean == pytest.approx(float(np.mean(eta.cpu().numpy())), rel=1e-12)
    sim.close()


@pytest.mark.parametrize("n", [1, 2, 3, 5, 33, 63, 64])
def test_edge_widths_eta_parity(n):
    require_cuda()
    rng = random.Random(500 + n)
    ops = []
    for _ in range(5 * n + 10):
        k = rng.randrange(4)
        if k == 0 or n == 1:
            ops.append(("H", rng.randrange(n)))
        elif k == 1:
            ops.append(("S", rng.randrange(n)))
        else:
            a, b = rng.sample(range(n), 2)
            ops.append(("CX" if k == 2 else "CZ", a, b))
    ops.insert(len(ops) // 2, ("T", rng.randrange(n)))
    ops.insert(len(ops) // 3, ("T", rng.randrange(n)))
    if n >= 3:
        ops.insert(len(ops) // 4, ("CCZ", 0, 1, 2))
    chi = 4 * (2 if n >= 3 else 1)
    sim = _sim(n, ops, chi, "exact")
    L = 40
    eta = _etas(sim, L, n)
    terms, coefs, _ = oracle_terms(n, ops, chi, "exact", parallel=n > 30)
    ov = oracle_overlaps(terms, coefs, n, n, L, parallel=True)
    _check(eta, ov, n, 1.0)
    sim.close()


def test_full_v_register():
    """|v| = 64 terms (H on every qubit)."""
    require_cuda()
    n = 64
    ops = [("H", q) for q in range(n)] + [("CZ", q, q + 1) for q in range(0, n - 1, 3)]
    ops += [("T", 7), ("S", 9)]
    sim = _sim(n, ops, 2, "exact")
    eta = _etas(sim, 32, 4)
    terms, coefs, _ = oracle_terms(n, ops, 2, "exact")
    ov = oracle_overlaps(terms, coefs, n, 4, 32, parallel=True)
    _check(eta, ov, n, 1.0)
    sim.close()


def test_mid_slice_eta_parity():
    """n=40, 2000 Cliffords + 24 T: 64 terms of the 2^16-term decomposition, L = 64."""
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, chi_total, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    alpha0, chi = 777, 64
    sim = _sim(n, ops, chi, "sparsify", seed=seed, alpha0=alpha0, chi_total=chi_total)
    L = 64
    eta = _etas(sim, L, 99)
    terms, coefs, _ = oracle_terms(n, ops, chi_total, "sparsify", seed=seed,
                                   alphas=range(alpha0, alpha0 + chi), parallel=True)
    ov = oracle_overlaps(terms, coefs, n, 99, L, parallel=True)
    _check(eta, ov, n, chi / chi_total)
    sim.close()


def test_hidden_shift_norm_is_one():
    """Exact 2^16-term decomposition of psi = |s>: every equatorial state has
    |<phi_A|s>|^2 = 2^-n, so eta_A = 1 for every A at full size."""
    require_cuda()
    cfg = workloads.config_hidden_shift()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    sim = _sim(n, ops, chi, "exact")
    eta, mean = sim.norm_estimate(256, seed=5, want_mean=True)
    e = eta.cpu().numpy()
    assert np.all(np.abs(e - 1.0) <= 1e-5), e[np.abs(e - 1.0) > 1e-5][:5]
    assert mean == pytest.approx(1.0, abs=1e-5)
    sim.close()


def test_fold_paths_agree_at_scale():
    """n=40 benchmark circuit, 4096 terms, L = 128: the change-of-variables path and
    the K path give the same eta to FP32 summation order."""
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, seed = cfg["n"], cfg["ops"], cfg["seed"]
    sim = _sim(n, ops, 4096, "sparsify", seed=seed, chi_total=cfg["chi"])
    e = _etas(sim, 128, 7)
    ref = e[-1]
    for f in FOLDS[1:]:
        assert np.all(np.abs(e[f] - ref) <= 1e-5 * np.maximum(np.abs(ref), 4096 / cfg["chi"])), f
    sim.close()


def test_qaoa_n50_slice_eta_vs_oracle_and_exact():
    """The n = 50 QAOA workload (gamma 0.3, beta 0.2; 2^20 sparsified terms): eta_l of a
    128-term slice on 16 equatorial states, against the FP64 oracle (both exact routes
    of the kernel) and the oracle's exact Z[zeta8] overlap sums."""
    require_cuda()
    from oracle import exact
    cfg = workloads.config_qaoa()
    n, ops, chi_total, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    alpha0, chi, L, aseed = 2 ** 19 + 1234, 128, 16, 99
    sim = _sim(n, ops, chi, "sparsify", seed=seed, alpha0=alpha0, chi_total=chi_total)
    terms, coefs, chs = oracle_terms(n, ops, chi_total, "sparsify", seed=seed,
                                     alphas=range(alpha0, alpha0 + chi), parallel=True)
    ov = oracle_overlaps(terms, coefs, n, aseed, L, parallel=True)
    norm2 = float(np.mean((2.0 ** n) * np.abs(ov) ** 2))
    _check(_etas(sim, L, aseed), ov, n, norm2)
    ex = exact.ExactDecomposition(n, ops, chi_total, "sparsify")
    got = sim.norm_estimate(L, seed=aseed).cpu().numpy()
    for l in range(4):
        want = float(ex.eta(terms, chs, E.draw_A(n, aseed, l)))
        assert abs(got[l] - want) <= 1e-5 * max(want, norm2)
    sim.close()
