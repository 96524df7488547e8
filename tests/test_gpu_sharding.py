"""Term-sharded estimators and chain checkpoints.  Every estimator of Sec. 4 is a sum
over terms: two contexts holding the two halves of the n = 40, 2^16-term decomposition
give the amplitudes and eta_l of one context holding all of it (partials summed before
anything is squared).  A chain's state is its string, the seed and the next step index
(the counter RNG draws depend on nothing else), so chains checkpointed after T1 steps
and resumed in a fresh context continue exactly as the uninterrupted chains."""
import numpy as np
import pytest
import torch

from paper_1808_00128_gb300 import lrstab, sharding, workloads
from tests._gpu import amp_tol, require_cuda

pytestmark = pytest.mark.gpu


def _ctx(low, n, chi, seed, a0=0, c=None, chi_total=None):
    s = lrstab.Simulator(n, 0)
    s.init_terms(low, c or chi, mode="sparsify", seed=seed, alpha0=a0, chi_total=chi_total or chi)
    s.apply_clifford(low.gates)
    return s


def test_sharded_amplitudes_and_eta_equal_full_context():
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, chi, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    low = lrstab.lower_circuit(n, ops)
    full = _ctx(low, n, chi, seed)
    shards = []
    for r in range(2):
        a0, c = sharding.shard_range(chi, r, 2)
        shards.append(_ctx(low, n, chi, seed, a0, c, chi))
    x = torch.cat([full.sample_terms(256, seed=3),
                   torch.from_numpy(workloads.random_bitstrings(n, 256, seed=4).view(np.int64)).cuda()])
    a_full = full.amplitude(x).cpu().numpy()
    a_sh = sharding.amplitude_sharded(shards, x).cpu().numpy()
    af, ash = a_full[:, 0] + 1j * a_full[:, 1], a_sh[:, 0] + 1j * a_sh[:, 1]
    assert np.all(np.abs(af - ash) <= amp_tol(af, n))
    L = 96
    e_full = full.norm_estimate(L, seed=77).cpu().numpy()
    e_sh = sharding.norm_estimate_sharded(shards, L, 77).cpu().numpy()
    np.testing.assert_allclose(e_sh, e_full, rtol=1e-5, atol=1e-5 * float(e_full.mean()))
    ov = full.norm_overlaps(L, 77)
    np.testing.assert_allclose(full.norm_eta_from_overlaps(ov).cpu().numpy(), e_full, rtol=1e-12)
    for s in shards + [full]:
        s.close()


def test_chain_checkpoint_and_resume():
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, chi, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    low = lrstab.lower_circuit(n, ops)
    C, T1, T2, mseed = 64, 16, 20, 31
    a = _ctx(low, n, chi, seed)
    x0 = a.sample_terms(C, seed=6)
    a.chains_init(x0)
    tr = torch.empty((T1 + T2, C), dtype=torch.int64, device="cuda:0")
    a.metropolis(T1 + T2, seed=mseed, trace=tr)
    # checkpoint after T1 steps: the strings (and P, not needed to resume)
    a.chains_init(x0)
    xc = torch.empty(C, dtype=torch.int64, device="cuda:0")
    a.metropolis(T1, seed=mseed, x_out=xc)
    ckpt = xc.cpu().numpy().copy()
    a.close()
    # resume in a fresh context from the checkpoint at global step T1
    b = _ctx(low, n, chi, seed)
    b.chains_init(torch.from_numpy(ckpt).cuda())
    tr2 = torch.empty((T2, C), dtype=torch.int64, device="cuda:0")
    b.metropolis(T2, seed=mseed, step0=T1, trace=tr2)
    assert np.array_equal(ckpt, tr[T1 - 1].cpu().numpy())
    assert torch.equal(tr2, tr[T1:])
    b.close()


def test_single_steps_continue_a_two_step_pass():
    """A two-step pass leaves up to two flips to commit; the one-step calls of the
    sharded protocol (propose, accept) that follow commit both, in order: one pass plus
    one propose/accept step equals three steps in one call (n = 50, 16-byte states)."""
    require_cuda()
    cfg = workloads.config_qaoa()
    n, ops, seed = cfg["n"], cfg["ops"], cfg["seed"]
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, 4096, mode="sparsify", seed=seed, chi_total=cfg["chi"])
    sim.apply_clifford(low.gates)
    assert sim.get_tuning("mc_lookahead") == 2
    C, mseed = 96, 17
    x0 = sim.sample_terms(C, seed=8)
    xa = torch.empty(C, dtype=torch.int64, device="cuda:0")
    tr = torch.empty((4, C), dtype=torch.int64, device="cuda:0")
    sim.chains_init(x0)
    sim.metropolis(4, seed=mseed, trace=tr, x_out=xa)
    # the same chains: one two-step pass, then steps 2 and 3 through propose / accept
    sim.chains_init(x0)
    sim.metropolis(2, seed=mseed)
    for step in (2, 3):
        amp = sim.metropolis_propose(mseed, step)
        row = torch.empty(C, dtype=torch.int64, device="cuda:0")
        sim.metropolis_accept(amp, mseed, step, trace=row)
        assert torch.equal(row, tr[step])
    xb = torch.empty(C, dtype=torch.int64, device="cuda:0")
    sim.metropolis(0, seed=mseed, step0=4, x_out=xb)
    assert torch.equal(xa, xb)
    assert int((tr[1] != x0).sum()) > 0           # moves were accepted in the pass
    sim.close()
