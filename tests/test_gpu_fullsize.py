"""Parity of the benchmark's full-size launches on sampled outputs.  The n = 50 QAOA
workload (2^20 sparsified terms) and the n = 40 workload (2^16) are launched as
bench.py launches them -- an amplitude batch of its 4096 strings, a norm estimate with
its L, Metropolis chains -- and sampled outputs are compared with the oracle's exact
Z[zeta8] sums over every term, computed by the C restatement of the oracle on all host
threads: amplitudes within 1e-5 max(|a|, ||psi|| 2^{-n/2}) and within the kernel's
stated bound, eta_l within 1e-5 max(eta, ||psi||^2), and chain decisions replayed with
the exact probabilities."""
import numpy as np
import pytest
import torch

from oracle import estimators as E
from oracle import fast
from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import require_cuda

pytestmark = pytest.mark.gpu

CASES = {
    "qaoa_n50_chi2^20": (workloads.config_qaoa, 512, 256),
    "clifford_t_n40_chi2^16": (workloads.config_mid, 256, 256),
}


@pytest.mark.parametrize("case", list(CASES))
def test_full_size_launch_vs_exact_oracle(case):
    require_cuda()
    make, L, C = CASES[case]
    cfg = make()
    n, ops, chi, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode="sparsify", seed=seed)
    sim.apply_clifford(low.gates)
    # the benchmark's amplitude batch; 32 of its outputs are checked
    xb = workloads.random_bitstrings(n, 4096, seed=workloads.SEED_BASE + 40)
    x = torch.from_numpy(xb.view(np.int64)).cuda()
    err = torch.empty(4096, dtype=torch.float32, device="cuda:0")
    amp = sim.amplitude(x, err=err).cpu().numpy()
    err = err.cpu().numpy().astype(np.float64)
    pick = np.linspace(0, 4095, 32).astype(int)
    # the benchmark's norm estimate; eta_0 and eta_1 are checked
    eta = sim.norm_estimate(L, seed=1000).cpu().numpy()
    norm2 = float(eta.mean())
    # chains as the benchmark starts them; 8 chains x 4 steps are replayed
    x0 = sim.sample_terms(C, seed=2000)
    sim.chains_init(x0)
    T, mseed = 4, 3000
    trace = torch.empty((T, C), dtype=torch.int64, device="cuda:0")
    sim.metropolis(T, seed=mseed, trace=trace)
    tr = trace.cpu().numpy().view(np.uint64)
    xs0 = x0.cpu().numpy().view(np.uint64)
    sim.close()
    chains = list(range(8))
    props, cur = [], xs0.copy()
    for t in range(T):
        for c in chains:
            j, _ = E.metropolis_draws(n, mseed, c, t)
            props.append(int(cur[c]) ^ (1 << j))
        cur = tr[t]
    strings = [int(xb[i]) for i in pick] + [int(xs0[c]) for c in chains] + props
    As = [E.draw_A(n, 1000, l) for l in range(2)]
    prep = fast.Prepared(n, ops, chi, "sparsify", seed)
    ex_amp, ex_ov = prep.sums(strings, As)
    ex_amp = np.array([fast.to_complex(z) for z in ex_amp])
    # amplitudes
    got = amp[pick, 0] + 1j * amp[pick, 1]
    want = ex_amp[:32]
    scale = np.maximum(np.abs(want), np.sqrt(norm2) * 2.0 ** (-n / 2))
    d = np.abs(got - want)
    assert np.all(d <= 1e-5 * scale), float((d / scale).max())
    assert np.all(d <= err[pick]), float((d / err[pick]).max())
    assert np.count_nonzero(np.abs(want) > 0) >= 16
    # equatorial states
    for l in range(2):
        e = fast.eta_of(ex_ov[l], n)
        assert abs(eta[l] - e) <= 1e-5 * max(e, norm2), (l, eta[l], e)
    # chain decisions with the exact probabilities
    P = {s: abs(a) ** 2 for s, a in zip(strings[32:], ex_amp[32:])}
    close = 0
    cur = xs0.copy()
    for t in range(T):
        for c in chains:
            x_, y_ = int(cur[c]), int(int(cur[c]) ^ (1 << E.metropolis_draws(n, mseed, c, t)[0]))
            _, r = E.metropolis_draws(n, mseed, c, t)
            acc = int(tr[t, c]) == y_
            assert acc or int(tr[t, c]) == x_
            px, py = P[x_], P[y_]
            if px <= 0 or py >= px:
                want_acc = True
            else:
                want_acc = r < py / px
                if abs(py / px - r) <= 1e-4 * (py / px):
                    close += 1
                    want_acc = acc
            assert acc == want_acc, (t, c)
        cur = tr[t]
    assert close <= 2


def test_hidden_shift_eight_term_ccz_chi_2_24_vs_exact_oracle():
    """The 40-qubit hidden shift with its 16 CCZ in the 8-term form (Eq.
    (CCZ_decomposition), prefactor 1/6, xi = 16/9) sparsified to chi = 2^24 terms (17 GB
    of tableau): <s|psi>, the amplitudes at the 40 neighbours of s and at random strings
    against the exact sums over all 2^24 terms; <s|psi> is 1 up to the sparsification
    error (delta^2 = ||c||_1^2 / chi = 5.9e-4)."""
    require_cuda()
    n, chi, dseed = 40, 1 << 24, 77
    ops, s = workloads.hidden_shift_circuit(n, 16, workloads.SEED_BASE + 3)
    low = lrstab.lower_circuit(n, ops, "sum8")
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode="sparsify", seed=dseed)
    sim.apply_clifford(low.gates)
    xs = [s] + [s ^ (1 << j) for j in range(n)] + [int(x) for x in workloads.random_bitstrings(n, 15, seed=9)]
    x = torch.tensor(np.asarray(xs, dtype=np.uint64).view(np.int64), device="cuda:0")
    err = torch.empty(len(xs), dtype=torch.float32, device="cuda:0")
    a = sim.amplitude(x, err=err).cpu().numpy()
    err = err.cpu().numpy().astype(np.float64)
    sim.close()
    got = a[:, 0] + 1j * a[:, 1]
    prep = fast.Prepared(n, ops, chi, "sparsify", dseed, ccz_mode="sum8")
    want = np.array([fast.to_complex(z) for z in prep.sums(xs)[0]])
    scale = np.maximum(np.abs(want), 2.0 ** (-n / 2))
    d = np.abs(got - want)
    assert np.all(d <= 1e-5 * scale), float((d / scale).max())
    assert np.all(d <= err)
    delta = np.sqrt(low.l1_norm ** 2 / chi)
    assert abs(abs(want[0]) - 1.0) <= 5 * delta
