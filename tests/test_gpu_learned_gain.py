"""What the trained proposal gains, measured in effective samples per second: on a
QAOA Max-E3LIN2 state small enough (n = 20) for its exact distribution P to be
enumerated, Metropolis-Hastings with the MADE proposal trained on single-flip chain
samples against the paper's single-flip chain (Sec. 4.2), both timed on the GPU and
both at the same accuracy against P."""
import pytest

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
