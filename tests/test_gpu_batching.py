"""Batched execution of several circuits of uneven chi in one persistent launch,
Metropolis steps replayed from a captured CUDA graph, and the launch-shape
autotuner: none of them may change results."""
import numpy as np
import pytest
import torch

from paper_1808_00128_gb300 import autotune, lrstab, workloads
from tests._gpu import amp_tol, require_cuda

pytestmark = pytest.mark.gpu


def test_batched_apply_matches_single_launches():
    require_cuda()
    n = 20
    sims, lows = [], []
    for i, chi in enumerate([300, 4096, 1000, 256 * 7]):     # uneven, ragged term counts
        ops, _ = workloads.qaoa_e3lin2_circuit(n, 4, 0.3, 0.2, seed=100 + i)
        low = lrstab.lower_circuit(n, ops)
        s = lrstab.Simulator(n, 0)
        s.init_terms(low, chi, mode="sparsify", seed=7 + i)
        sims.append(s)
        lows.append(low)
    lrstab.apply_clifford_batch(sims, [l.gates for l in lows])
    for i, (s, low) in enumerate(zip(sims, lows)):
        ref = lrstab.Simulator(n, 0)
        ref.init_terms(low, s.chi, mode="sparsify", seed=7 + i)
        ref.apply_clifford(low.gates)
        a, b = s.export_terms(), ref.export_terms()
        for k in ("F", "G", "M", "gamma", "v", "s", "omega", "coef", "choice"):
            assert np.array_equal(a[k], b[k]), (i, k)
        ref.close()
    for s in sims:
        s.close()


def test_tuning_knobs_keep_results():
    require_cuda()
    cfg = workloads.config_mid()
    n, ops = cfg["n"], cfg["ops"]
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, 1 << 14, mode="sparsify", seed=cfg["seed"], chi_total=1 << 16)
    sim.apply_clifford(low.gates)
    x = torch.cat([sim.sample_terms(700, seed=3),
                   torch.from_numpy(workloads.random_bitstrings(n, 300, 4).view(np.int64)).cuda()])
    base = sim.amplitude(x).cpu().numpy()
    eta0 = sim.norm_estimate(96, seed=5).cpu().numpy()
    want = base[:, 0] + 1j * base[:, 1]
    for v in (1, 3, 32):
        sim.set_tuning("amp_blocks_per_sm", v)
        got = sim.amplitude(x).cpu().numpy()
        assert np.all(np.abs(got[:, 0] + 1j * got[:, 1] - want) <= amp_tol(want, n, 0.5))
    for v in (64, 512, 4096):
        sim.set_tuning("norm_max_tiles", v)
        eta = sim.norm_estimate(96, seed=5).cpu().numpy()
        assert np.all(np.abs(eta - eta0) <= 1e-5 * np.maximum(eta0, 0.25))
    with pytest.raises(lrstab.LrsError):
        sim.set_tuning("mc_chains_per_block", 65)
    # chains per block and chains in flight per block: same trajectory
    x0 = sim.sample_terms(100, seed=9)
    outs = []
    for cg, st in ((64, 2), (7, 2), (64, 1), (13, 3), (64, 4)):
        sim.set_tuning("mc_chains_per_block", cg)
        sim.set_tuning("mc_stages", st)
        sim.chains_init(x0)
        xo = torch.empty(100, dtype=torch.int64, device="cuda:0")
        sim.metropolis(40, seed=2, x_out=xo)     # 40 steps: two graph replays + 8 direct steps
        outs.append(xo.cpu())
    for o in outs[1:]:
        assert torch.equal(outs[0], o)
    with pytest.raises(lrstab.LrsError):
        sim.set_tuning("mc_stages", 5)
    sim.set_tuning("mc_chains_per_block", 7)
    sim.set_tuning("mc_stages", 2)
    chosen = autotune.tune(sim, x=x, L=64, chains=100)
    assert set(chosen) == {"amp_blocks_per_sm", "norm_max_tiles", "norm_max_folds", "mc_chains_per_block",
                           "mc_stages", "mc_lookahead"}
    for k, (v, ms) in chosen.items():
        assert v in autotune.CANDIDATES[k] and ms > 0
        assert sim.get_tuning(k) == v
    sim.close()


def test_batched_amplitudes_equal_single_calls_and_oracle():
    """Four circuits of uneven chi (ragged term counts, one empty batch) in one batched
    amplitude launch and one reduction: each equals its own lrs_amplitude call bit for
    bit, and the smallest equals the oracle within the amplitude tolerance."""
    require_cuda()
    from oracle import estimators as E
    from tests._gpu import oracle_terms
    n = 14
    sims, xs, specs = [], [], []
    for i, (chi, B) in enumerate([(300, 37), (4096, 2048), (1000, 0), (256 * 7 + 5, 777)]):
        ops, _ = workloads.qaoa_e3lin2_circuit(n, 4, 0.3, 0.2, seed=200 + i)
        low = lrstab.lower_circuit(n, ops)
        s = lrstab.Simulator(n, 0)
        s.init_terms(low, chi, mode="sparsify", seed=9 + i)
        s.apply_clifford(low.gates)
        sims.append(s)
        specs.append((ops, chi, 9 + i))
        xs.append(torch.from_numpy(workloads.random_bitstrings(n, B, seed=50 + i).view(np.int64)).cuda())
    outs = lrstab.amplitude_batch(sims, xs)
    for s, x, o in zip(sims, xs, outs):
        assert torch.equal(o, s.amplitude(x))
    ops, chi, seed = specs[0]
    terms, coefs, _ = oracle_terms(n, ops, chi, "sparsify", seed=seed, parallel=True)
    got = outs[0].cpu().numpy()
    got = got[:, 0] + 1j * got[:, 1]
    want = np.array([E.amplitude(terms, coefs, int(x)) for x in xs[0].cpu().numpy().view(np.uint64)])
    assert np.all(np.abs(got - want) <= amp_tol(want, n, abs(coefs[0]) * np.sqrt(chi)))
    with pytest.raises(lrstab.LrsError):
        lrstab.amplitude_batch([sims[0], sims[0]], [xs[0], xs[0]])
    for s in sims:
        s.close()


def test_create_with_options():
    """lrs_options: initial knobs as lrs_set_tuning would set them, defaults for the
    rest; a value lrs_set_tuning rejects or a short struct fails the create."""
    require_cuda()
    sim = lrstab.Simulator(50, 0, tuning={"apply_lanes": 2, "mc_lookahead": 1, "norm_max_folds": -1})
    assert sim.get_tuning("apply_lanes") == 2
    assert sim.get_tuning("mc_lookahead") == 1
    assert sim.get_tuning("norm_max_folds") == -1
    assert sim.get_tuning("mc_stages") == 1            # default
    sim.close()
    with pytest.raises(lrstab.LrsError):
        lrstab.Simulator(50, 0, tuning={"apply_lanes": 3})
    o = lrstab.options({"mc_stages": 2})
    o.size = 8
    h = lrstab.C.c_void_p()
    rc = lrstab.lib().lrs_create(0, 50, lrstab.C.byref(o), lrstab.C.byref(h))
    assert rc == -1 and not h.value
