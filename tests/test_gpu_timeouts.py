"""Failure paths of the bounded device waits.  A one-shot test request makes one block
of the next Metropolis propose launch, or of the next tcgen05 GEMM, expect 16 bytes
more than its copies deliver; that block's wait runs out after 1 s, it waits for its
own copies, frees what it holds and returns.  The next synchronising call must report
LRS_ERR_TIMEOUT, and the calls after it must run normally and reproduce the results of
a run without the request.  Nothing faults: the copies all land, every wait is bounded."""
import numpy as np
import pytest
import torch

from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import require_cuda

pytestmark = pytest.mark.gpu

TIMEOUT = -4


def _chains(sim, x0, steps, seed):
    xo = torch.empty(x0.numel(), dtype=torch.int64, device="cuda:0")
    po = torch.empty(x0.numel(), dtype=torch.float64, device="cuda:0")
    sim.chains_init(x0)
    sim.metropolis(steps, seed=seed, x_out=xo, p_out=po)
    torch.cuda.synchronize()
    return xo.cpu().numpy(), po.cpu().numpy()


@pytest.mark.parametrize("steps", [1, 16])   # one direct launch; one graph replay
def test_metropolis_wait_runs_out_then_recovers(steps):
    require_cuda()
    cfg = workloads.config_tiny()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode="exact")
    sim.apply_clifford(low.gates)
    x0 = sim.sample_terms(32, seed=3)
    want = _chains(sim, x0, steps, seed=11)
    sim.debug_inject_wait_timeout()
    sim.chains_init(x0)
    sim.metropolis(steps, seed=11)           # enqueued; one block's wait runs out
    torch.cuda.synchronize()
    with pytest.raises(lrstab.LrsError) as e:
        sim.metropolis(1, seed=11, step0=steps)
    assert e.value.status == TIMEOUT
    got = _chains(sim, x0, steps, seed=11)   # recovers: same chains as without the request
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1])
    sim.close()


def test_tcgen05_gemm_wait_runs_out_then_recovers():
    require_cuda()
    n, H, B = 20, 256, 1024
    net = lrstab.MLP(n, H, 0)
    rng = np.random.default_rng(1)
    net.set_params(dict(W1=rng.uniform(-0.2, 0.2, (H, n)), b1=rng.uniform(-0.2, 0.2, H),
                        W2=rng.uniform(-0.06, 0.06, (H, H)), b2=rng.uniform(-0.06, 0.06, H),
                        W3=rng.uniform(-0.06, 0.06, (n, H)), b3=rng.uniform(-0.06, 0.06, n)))
    assert net.gemm == lrstab.MLP.GEMM_TCGEN05
    x = torch.from_numpy(workloads.random_bitstrings(n, B, seed=2).view(np.int64)).cuda()
    want = net.forward(x)[0].cpu().numpy()
    net.debug_inject_wait_timeout()
    net.forward(x)
    torch.cuda.synchronize()
    with pytest.raises(lrstab.LrsError) as e:
        net.get_params()
    assert e.value.status == TIMEOUT
    net.get_params()                          # the flag is cleared
    got = net.forward(x)[0].cpu().numpy()
    net.get_params()
    assert np.array_equal(got, want)
    # without a synchronising call: the flag reaches the host with the call's own
    # asynchronous copy, and the next enqueuing call reports it
    net.debug_inject_wait_timeout()
    net.forward(x)
    torch.cuda.synchronize()
    with pytest.raises(lrstab.LrsError) as e:
        net.forward(x)
    assert e.value.status == TIMEOUT
    got = net.forward(x)[0].cpu().numpy()
    net.get_params()
    assert np.array_equal(got, want)
    net.close()
