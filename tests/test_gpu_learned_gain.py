"""What the trained proposal gains: on a QAOA Max-E3LIN2 state small enough for
its exact distribution P to be enumerated, Metropolis-Hastings with the MADE
proposal trained on single-flip chain samples decorrelates far faster per step
than the paper's single-flip chain (Sec. 4.2), at the same accuracy against P."""
import pytest

from tests._gpu import require_cuda

pytestmark = pytest.mark.gpu


def test_learned_proposal_beats_single_flip():
    require_cuda()
    import bench
    r = bench.sampler_study(n=14, chi=1 << 12, C=512, T_plain=1500, T_learned=150, hidden=256,
                            train_steps=400)
    p, l = r["plain"], r["learned"]
    # both samplers reproduce P on the cost and Hamming-weight histograms
    assert p["tv_cost"] < 0.03 and l["tv_cost"] < 0.03
    assert p["tv_hamming"] < 0.03 and l["tv_hamming"] < 0.03
    # the network learned P: its NLL is close to the entropy of P
    assert l["nll"] < l["entropy_of_P"] + 0.5
    # effective samples per step: at least 3x the single-flip chain
    assert p["tau_int"] / l["tau_int"] > 3.0
    assert l["acceptance"] > 0.3
