"""A whole step of several circuits captured into one CUDA graph: re-initialised terms
(Lemma (Sparsification) choices drawn again), batched gate updates, batched amplitudes
(Eq. (amplitude)), norm estimates (Sec. 4.3), chain starts and Metropolis steps
(Sec. 4.2) of two n = 50 QAOA circuits with chi = 2^14 and 2^15.  The graph's replays
give, bit for bit, what the uncaptured calls give (every kernel is deterministic and
takes its seeds at capture)."""
import numpy as np
import pytest
import torch

from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import require_cuda

pytestmark = pytest.mark.gpu


def test_step_of_two_circuits_replays_bit_for_bit():
    require_cuda()
    dev = torch.device("cuda:0")
    chis, B, L, C, T = [1 << 14, 1 << 15], 512, 64, 96, 20   # T > 16: graph-sized Metropolis runs
    sims, lows = [], []
    for i, chi in enumerate(chis):
        ops, _ = workloads.qaoa_e3lin2_circuit(50, 4, 0.3, 0.2, workloads.SEED_BASE + 4 + i)
        low = lrstab.lower_circuit(50, ops)
        s = lrstab.Simulator(50, 0)
        s.init_terms(low, chi, mode="sparsify", seed=workloads.SEED_BASE + 14 + i)
        sims.append(s)
        lows.append(low)
    xs = [torch.from_numpy(workloads.random_bitstrings(50, B, seed=workloads.SEED_BASE + 70 + i).view(np.int64))
          .to(dev) for i in range(len(sims))]
    amps = [torch.empty((B, 2), dtype=torch.float64, device=dev) for _ in sims]
    etas = [torch.empty(L, dtype=torch.float64, device=dev) for _ in sims]
    x0s = [torch.empty(C, dtype=torch.int64, device=dev) for _ in sims]
    xos = [torch.empty(C, dtype=torch.int64, device=dev) for _ in sims]
    pos = [torch.empty(C, dtype=torch.float64, device=dev) for _ in sims]
    outs = amps + etas + x0s + xos + pos

    def step():
        for i, s in enumerate(sims):
            s.reinit_terms(seed=workloads.SEED_BASE + 14 + i)
        lrstab.apply_clifford_batch(sims, [l.gates for l in lows])
        lrstab.amplitude_batch(sims, xs, amps)
        for i, s in enumerate(sims):
            s.norm_estimate(L, seed=200 + i, eta=etas[i])
            s.sample_terms(C, seed=300 + i, x=x0s[i])
            s.chains_init(x0s[i])
            s.metropolis(T, seed=400 + i, x_out=xos[i], p_out=pos[i])

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()                               # sizes every buffer, sets kernel attributes
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    torch.cuda.synchronize()
    for rep in range(2):
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(ref, outs):
            assert torch.equal(a, b), rep
    assert all(int((x != x0).sum()) > 0 for x, x0 in zip(xos, x0s))   # the chains moved
    assert all(float(e.mean()) > 0.5 for e in etas)
    g.reset()
    for s in sims:
        s.close()


def test_reinit_terms_equals_init_terms():
    """lrs_reinit_terms from the tables on the device equals a fresh lrs_init_terms with
    the same seed (every tableau word, phase and coefficient), also for a context whose
    terms came from lrs_copy_terms."""
    require_cuda()
    cfg = workloads.config_mid()
    n = cfg["n"]
    low = lrstab.lower_circuit(n, cfg["ops"])
    a = lrstab.Simulator(n, 0)
    b = lrstab.Simulator(n, 0)
    c = lrstab.Simulator(n, 0)
    a.init_terms(low, 3000, mode="sparsify", seed=11)
    b.init_terms(low, 3000, mode="sparsify", seed=12)
    b.apply_clifford(low.gates)
    b.reinit_terms(seed=11)
    c.copy_terms_from(b)
    c.apply_clifford(low.gates)
    c.reinit_terms(seed=11)
    ea, eb, ec = a.export_terms(), b.export_terms(), c.export_terms()
    for k in ea:
        assert np.array_equal(ea[k], eb[k]), k
        assert np.array_equal(ea[k], ec[k]), k
    d = lrstab.Simulator(n, 0)
    with pytest.raises(lrstab.LrsError):
        d.reinit_terms(seed=1)                # no terms yet
    for s in (a, b, c, d):
        s.close()
