"""The allocation-free amplitude entry point (for callers that cannot call
cudaMalloc when they need amplitudes) must return what lrs_amplitude returns,
call after call, while using its fixed device buffer.  This file sorts last so
that a failure here comes after every other test has run."""
import numpy as np
import pytest
import torch

from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import amp_tol, require_cuda

pytestmark = pytest.mark.gpu


def test_noalloc_matches_amplitude_twice():
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, chi, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode="sparsify", seed=seed)
    sim.apply_clifford(low.gates)
    xt = sim.sample_terms(2048, seed=21)
    xr = torch.from_numpy(workloads.random_bitstrings(n, 2048, seed=22).view(np.int64)).cuda()
    x = torch.cat([xt, xr])                       # 4096 strings: the largest batch at chi = 2^16
    ref = sim.amplitude(x).cpu().numpy()
    want = ref[:, 0] + 1j * ref[:, 1]
    for call in range(2):
        out = torch.full((x.numel(), 2), float("nan"), dtype=torch.float64, device="cuda:0")
        sim.amplitude_noalloc(x, out)
        got = out.cpu().numpy()
        got = got[:, 0] + 1j * got[:, 1]
        assert np.all(np.abs(got - want) <= amp_tol(want, n)), f"call {call}"
    # a second batch through the same fixed buffer after the first
    y = x[:1000].flip(0).contiguous()
    out = torch.empty((1000, 2), dtype=torch.float64, device="cuda:0")
    sim.amplitude_noalloc(y, out)
    ref2 = sim.amplitude(y).cpu().numpy()
    np.testing.assert_allclose(out.cpu().numpy(), ref2, rtol=0, atol=float(amp_tol(np.zeros(1), n)[0]))
    with pytest.raises(lrstab.LrsError):
        nb = (1 << 21) + 1                        # more partial sums than the fixed buffer holds
        big = torch.zeros(nb, dtype=torch.int64, device="cuda:0")
        sim.amplitude_noalloc(big, torch.empty((nb, 2), dtype=torch.float64, device="cuda:0"))
    sim.close()
