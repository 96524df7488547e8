"""What the trained proposal gains, measured in effective samples per second: on a
QAOA Max-E3LIN2 state small enough (n = 20) for its exact distribution P to be
enumerated, Metropolis-Hastings with the MADE proposal trained on single-flip chain
samples against the paper's single-flip chain (Sec. 4.2), both timed on the GPU and
both at the same accuracy against P; and on the hidden shift, where single flips cannot
find the shift at all."""
import numpy as np
import pytest
import torch

from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import require_cuda

pytestmark = pytest.mark.gpu


def test_learned_proposal_beats_single_flip_in_ess_per_second():
    require_cuda()
    import bench
    r = bench.sampler_study(n=20, chi=1 << 14, C=1024, hidden=512, train_samples=60_000, epochs=8,
                            plain_steps=800, learned_steps=120, burn=100, tv_targets=(0.05,))
    p, l = r["plain"], r["learned"]
    # both samplers reach the same accuracy against P (cost histogram and bit marginals)
    assert r["matched_tv"]["0.05"]["plain_gpu_s"] is not None
    assert r["matched_tv"]["0.05"]["learned_gpu_s"] is not None
    assert l["tv_cost_end"] < 0.05 and p["tv_cost_end"] < 0.05
    # effective samples per GPU second of sampling: the learned proposal is ahead
    assert r["ess_ratio_learned_over_plain"] > 1.2
    # with the plain steps that made its training data and the training charged, it is
    # ahead beyond a finite number of effective samples
    assert r["breakeven_effective_samples"] is not None and r["breakeven_effective_samples"] > 0
    assert l["acceptance"] > 0.3


def test_hidden_shift_term_sampled_chains():
    """Config 3's chains: started at strings sampled from single terms, single flips do
    not find the shift s (P = |<x|psi>|^2 is 0 at every string but s, so a flip chain
    walks blindly); the learned proposal trained on the chain-rule marginal sampler's
    exact samples (end of Sec. 4.3) takes every chain to s, where it stays."""
    require_cuda()
    cfg = workloads.config_hidden_shift()
    n, chi, s = cfg["n"], cfg["chi"], int(cfg["shift"])
    low = lrstab.lower_circuit(n, cfg["ops"])
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode="exact")
    sim.apply_clifford(low.gates)
    C = 256
    x0 = sim.sample_terms(C, seed=31)
    started = int((x0 == s).sum().item())
    sim.chains_init(x0)
    xo = torch.empty(C, dtype=torch.int64, device="cuda:0")
    sim.metropolis(64, seed=41, x_out=xo)
    assert int((xo == s).sum().item()) <= started + 2
    work = (lrstab.Simulator(n, 0), lrstab.Simulator(n, 0))
    bits, _ = sim.marginal_sample(list(range(n)), 256, 3, seed=100, work=work)
    for w_ in work:
        w_.close()
    sample = sum(int(b) << q for q, b in enumerate(bits))
    assert sample == s
    H = 512
    net = lrstab.MLP(n, H, 0)
    rng = np.random.default_rng(5)
    l1, l2 = 1 / np.sqrt(n), 1 / np.sqrt(H)
    net.set_params(dict(W1=rng.uniform(-l1, l1, (H, n)), b1=rng.uniform(-l1, l1, H),
                        W2=rng.uniform(-l2, l2, (H, H)), b2=rng.uniform(-l2, l2, H),
                        W3=rng.uniform(-l2, l2, (n, H)), b3=rng.uniform(-l2, l2, n)))
    data = torch.full((1024,), sample, dtype=torch.int64, device="cuda:0")
    for _ in range(500):
        net.train_step(data, lr=1e-3)
    sim.chains_init(x0)
    po = torch.empty(C, dtype=torch.float64, device="cuda:0")
    lrstab.metropolis_learned(sim, net, 32, seed=43, x_out=xo, p_out=po)
    at = (xo == s).cpu().numpy()
    assert at.sum() >= 0.99 * C                 # an independent proposal with q(s) near 1
    assert np.allclose(po.cpu().numpy()[at], 1.0, atol=1e-5)
    net.close()
    sim.close()
