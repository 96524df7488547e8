"""Metropolis parity (Sec. 4.2): CUDA chains replayed step by step by the oracle
on the same counter-RNG draws.  A decision may differ only when the FP64 ratio
sits within 1e-4 (relative) of the uniform draw; the oracle then follows the
CUDA chain."""
import numpy as np
import pytest
import torch

from oracle import estimators as E
from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import oracle_terms, require_cuda

pytestmark = pytest.mark.gpu


def _sim(n, ops, chi, mode, seed=0):
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode=mode, seed=seed)
    sim.apply_clifford(low.gates)
    return sim


@pytest.mark.parametrize("case", ["tiny_exact", "sparse_ragged"])
def test_chain_replay(case):
    require_cuda()
    if case == "tiny_exact":
        cfg = workloads.config_tiny()
        n, ops, chi, mode, seed = cfg["n"], cfg["ops"], cfg["chi"], "exact", 0
    else:
        n, chi, mode, seed = 12, 600, "sparsify", 3
        ops = workloads.random_clifford_t(n, 220, 10, seed=71)
    sim = _sim(n, ops, chi, mode, seed)
    C, T, mseed = 70, 25, 1234
    x0 = sim.sample_terms(C, seed=8)
    sim.chains_init(x0)
    trace = torch.empty((T, C), dtype=torch.int64, device="cuda:0")
    pout = torch.empty(C, dtype=torch.float64, device="cuda:0")
    sim.metropolis(T, seed=mseed, trace=trace, p_out=pout)
    trace = trace.cpu().numpy().view(np.uint64)
    pout = pout.cpu().numpy()
    x0 = x0.cpu().numpy().view(np.uint64)
    terms, coefs, _ = oracle_terms(n, ops, chi, mode, seed=seed, parallel=chi > 100)
    close_calls = 0
    for c in range(C):
        x = int(x0[c])
        px = E.probability(terms, coefs, x)
        for t in range(T):
            j, r = E.metropolis_draws(n, mseed, c, t)
            y = x ^ (1 << j)
            py = E.probability(terms, coefs, y)
            gpu_acc = int(trace[t, c]) == y
            if not gpu_acc:
                assert int(trace[t, c]) == x, f"chain {c} step {t}: not x or y"
            if py >= px:
                want = True
            else:
                ratio = py / px
                want = r < ratio
                if abs(ratio - r) <= 1e-4 * ratio:
                    close_calls += 1
                    want = gpu_acc
            assert gpu_acc == want, f"chain {c} step {t}: P(y)/P(x) decision differs"
            if want:
                x, px = y, py
        assert abs(pout[c] - px) <= 1e-5 * max(px, 2.0 ** (-n)) * 2 + 1e-300
    assert close_calls < C * T // 50


def test_metropolis_continuation_and_errors():
    """Two calls of T/2 steps equal one call of T steps (pending flips persist)."""
    require_cuda()
    cfg = workloads.config_tiny()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    sim = _sim(n, ops, chi, "exact")
    C = 32
    x0 = sim.sample_terms(C, seed=2)
    xa = torch.empty(C, dtype=torch.int64, device="cuda:0")
    xb = torch.empty(C, dtype=torch.int64, device="cuda:0")
    sim.chains_init(x0)
    sim.metropolis(20, seed=5, x_out=xa)
    sim.chains_init(x0)
    sim.metropolis(10, seed=5, step0=0)
    sim.metropolis(10, seed=5, step0=10, x_out=xb)
    assert torch.equal(xa, xb)
    with pytest.raises(lrstab.LrsError):
        sim.metropolis(-1, seed=0)
    sim.close()
