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


@pytest.mark.parametrize("case", ["tiny_exact", "sparse_ragged", "wide_16_byte_states"])
def test_chain_replay(case):
    """Chains on 12-byte Pauli states (n <= 40) and on 16-byte ones (n = 44)."""
    require_cuda()
    C, T, mseed = 70, 25, 1234
    if case == "tiny_exact":
        cfg = workloads.config_tiny()
        n, ops, chi, mode, seed = cfg["n"], cfg["ops"], cfg["chi"], "exact", 0
    elif case == "sparse_ragged":
        n, chi, mode, seed = 12, 600, "sparsify", 3
        ops = workloads.random_clifford_t(n, 220, 10, seed=71)
    else:
        n, chi, mode, seed = 44, 32, "exact", 0
        ops = workloads.random_clifford_t(n, 300, 5, seed=72)
        C, T = 24, 12
    sim = _sim(n, ops, chi, mode, seed)
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
    # odd splits: a two-step pass's second pending flip carries into a single step and
    # into the next call
    for look in (1, 2):
        sim.set_tuning("mc_lookahead", look)
        sim.chains_init(x0)
        sim.metropolis(7, seed=5, step0=0)
        sim.metropolis(13, seed=5, step0=7, x_out=xb)
        assert torch.equal(xa, xb), look
    with pytest.raises(lrstab.LrsError):
        sim.set_tuning("mc_lookahead", 3)
    with pytest.raises(lrstab.LrsError):
        sim.metropolis(-1, seed=0)
    sim.close()


@pytest.mark.parametrize("chi,C", [(1 << 16, 64), (1 << 24, 8)], ids=["chi65536", "chi16777216_tiles_on_x"])
def test_full_size_chains_match_amplitudes(chi, C):
    """n=40 benchmark circuit at full size (2^16 terms, 64 chains) and sparsified to
    2^24 terms (8 chains: 65536 term tiles, more than the grid's y limit, so the tiles
    run along x), 32 steps (two graph replays): every decision replayed with
    P = |<x|psi>|^2 from the amplitude kernel (oracle-checked on slices), and the
    incremental P(x) of every chain equal to the amplitude kernel's at the end."""
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, seed = cfg["n"], cfg["ops"], cfg["seed"]
    sim = _sim(n, ops, chi, "sparsify", seed)
    T, mseed = 32, 99
    x0 = sim.sample_terms(C, seed=12)
    sim.chains_init(x0)
    xo = torch.empty(C, dtype=torch.int64, device="cuda:0")
    po = torch.empty(C, dtype=torch.float64, device="cuda:0")
    sim.metropolis(T, seed=mseed, x_out=xo, p_out=po)          # graph-replayed steps
    sim.chains_init(x0)
    trace = torch.empty((T, C), dtype=torch.int64, device="cuda:0")
    sim.metropolis(T, seed=mseed, trace=trace)                  # direct steps
    assert torch.equal(trace[-1], xo)
    tr = trace.cpu().numpy().view(np.uint64)
    xs = x0.cpu().numpy().view(np.uint64)
    # proposals of every step, from the same draws as the kernels
    props = np.zeros((T, C), np.uint64)
    cur = xs.copy()
    for t in range(T):
        for c in range(C):
            j, _ = E.metropolis_draws(n, mseed, c, t)
            props[t, c] = np.uint64(int(cur[c]) ^ (1 << j))
        cur = tr[t]
    allx = np.concatenate([xs, props.reshape(-1)])
    amp = sim.amplitude(torch.from_numpy(allx.view(np.int64)).cuda()).cpu().numpy()
    P = amp[:, 0] ** 2 + amp[:, 1] ** 2
    pmap = dict(zip(allx.tolist(), P.tolist()))
    close = 0
    cur = xs.copy()
    for t in range(T):
        for c in range(C):
            x, y = int(cur[c]), int(props[t, c])
            px, py = pmap[x], pmap[y]
            _, r = E.metropolis_draws(n, mseed, c, t)
            acc = int(tr[t, c]) == y
            assert acc or int(tr[t, c]) == x
            if px <= 0 or py >= px:
                want = True
            else:
                want = r < py / px
                if abs(py / px - r) <= 1e-4 * (py / px):
                    close += 1
                    want = acc
            assert acc == want, (t, c)
        cur = tr[t]
    final = sim.amplitude(xo).cpu().numpy()
    pf = final[:, 0] ** 2 + final[:, 1] ** 2
    np.testing.assert_allclose(po.cpu().numpy(), pf, rtol=1e-5, atol=1e-12 * pf.max())
    assert close < C * T // 50
    sim.close()


def test_hidden_shift_chains_stay_at_the_shift():
    """The n=40 hidden shift with its exact 2^16-term decomposition and 1024 chains (the
    chain count of that workload) started at the shift s: |<x|psi>|^2 is 1 at s and 0
    elsewhere, so every proposal is rejected, and the chains keep x = s, P(s) = 1."""
    require_cuda()
    cfg = workloads.config_hidden_shift()
    n, ops, chi, s = cfg["n"], cfg["ops"], cfg["chi"], cfg["shift"]
    C = cfg["chains"]
    assert C == 1024
    sim = _sim(n, ops, chi, "exact")
    x0 = torch.full((C,), int(s), dtype=torch.int64, device="cuda:0")   # s < 2^40
    sim.chains_init(x0)
    xo = torch.empty(C, dtype=torch.int64, device="cuda:0")
    po = torch.empty(C, dtype=torch.float64, device="cuda:0")
    sim.metropolis(32, seed=4, x_out=xo, p_out=po)
    xo = xo.cpu().numpy().view(np.uint64)
    po = po.cpu().numpy()
    assert np.all(xo == np.uint64(s))
    assert np.all(np.abs(po - 1.0) <= 1e-5)
    sim.close()


def test_chain_replay_qaoa_n50_slice():
    """Chains on 16-byte Pauli states at the QAOA workload's width (n = 50, gamma 0.3,
    beta 0.2): a 256-term slice of its 2^20-term sparsified decomposition, 24 chains x
    20 steps replayed decision by decision by the oracle."""
    require_cuda()
    cfg = workloads.config_qaoa()
    n, ops, chi_total, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    alpha0, chi, C, T, mseed = 4096, 256, 24, 20, 4321
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode="sparsify", seed=seed, alpha0=alpha0, chi_total=chi_total)
    sim.apply_clifford(low.gates)
    x0 = sim.sample_terms(C, seed=9)
    sim.chains_init(x0)
    trace = torch.empty((T, C), dtype=torch.int64, device="cuda:0")
    pout = torch.empty(C, dtype=torch.float64, device="cuda:0")
    sim.metropolis(T, seed=mseed, trace=trace, p_out=pout)
    trace = trace.cpu().numpy().view(np.uint64)
    pout = pout.cpu().numpy()
    x0 = x0.cpu().numpy().view(np.uint64)
    terms, coefs, _ = oracle_terms(n, ops, chi_total, "sparsify", seed=seed,
                                   alphas=range(alpha0, alpha0 + chi), parallel=True)
    close, moves = 0, 0
    for c in range(C):
        x = int(x0[c])
        px = E.probability(terms, coefs, x)
        for t in range(T):
            j, r = E.metropolis_draws(n, mseed, c, t)
            y = x ^ (1 << j)
            py = E.probability(terms, coefs, y)
            acc = int(trace[t, c]) == y
            assert acc or int(trace[t, c]) == x
            if px <= 0 or py >= px:
                want = True
            else:
                want = r < py / px
                if abs(py / px - r) <= 1e-4 * (py / px):
                    close += 1
                    want = acc
            assert acc == want, (c, t)
            if want:
                x, px = y, py
                moves += 1
        assert abs(pout[c] - px) <= 1e-5 * max(px, 1e-300) + 1e-300
    assert close < C * T // 50
    assert moves > 0
    sim.close()


def test_term_sharded_chains_equal_full_context():
    """Two contexts holding the two halves of the n = 40, 2^16-term decomposition run
    the chains through lrs_metropolis_propose / sum / lrs_metropolis_accept; the chains
    equal those of one context holding all terms (same draws, same decisions), and the
    final P(x) agree to FP32 summation accuracy."""
    require_cuda()
    from paper_1808_00128_gb300 import sharding
    cfg = workloads.config_mid()
    n, ops, chi, seed = cfg["n"], cfg["ops"], cfg["chi"], cfg["seed"]
    low = lrstab.lower_circuit(n, ops)
    full = lrstab.Simulator(n, 0)
    full.init_terms(low, chi, mode="sparsify", seed=seed)
    full.apply_clifford(low.gates)
    shards = []
    for r in range(2):
        a0, c = sharding.shard_range(chi, r, 2)
        s = lrstab.Simulator(n, 0)
        s.init_terms(low, c, mode="sparsify", seed=seed, alpha0=a0, chi_total=chi)
        s.apply_clifford(low.gates)
        shards.append(s)
    C, T, mseed = 48, 24, 777
    x0 = full.sample_terms(C, seed=5)
    full.chains_init(x0)
    tr_full = torch.empty((T, C), dtype=torch.int64, device="cuda:0")
    pf = torch.empty(C, dtype=torch.float64, device="cuda:0")
    full.metropolis(T, seed=mseed, trace=tr_full, p_out=pf)
    sharding.chains_init_sharded(shards, x0)
    tr = torch.empty((T, C), dtype=torch.int64, device="cuda:0")
    sharding.metropolis_sharded(shards, T, mseed, trace=tr)
    assert torch.equal(tr, tr_full)
    ps = torch.empty(C, dtype=torch.float64, device="cuda:0")
    shards[0].metropolis(0, seed=mseed, step0=T, p_out=ps)
    np.testing.assert_allclose(ps.cpu().numpy(), pf.cpu().numpy(), rtol=1e-5)
    with pytest.raises(lrstab.LrsError):
        shards[0].metropolis_accept(torch.zeros((C, 2), dtype=torch.float64, device="cuda:0"), mseed, T + 5)
    for s in shards + [full]:
        s.close()


@pytest.mark.parametrize("case", ["n40_12_byte_states", "qaoa_n50_16_byte_states"])
def test_two_step_passes_equal_single_steps(case):
    """Two steps per pass over the Pauli states (the default) against one step per
    pass: the same chains bit for bit -- every trace row, final string and P(x) --
    with ragged chain groups (70 chains), an odd step count with a trace (no graph) and
    one with graph replays and a leftover single step."""
    require_cuda()
    cfg = workloads.config_mid() if case.startswith("n40") else workloads.config_qaoa()
    n, ops = cfg["n"], cfg["ops"]
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, 8192, mode="sparsify", seed=cfg["seed"], chi_total=cfg["chi"])
    sim.apply_clifford(low.gates)
    C = 70
    x0 = sim.sample_terms(C, seed=4)
    res = {}
    for look in (1, 2):
        sim.set_tuning("mc_lookahead", look)
        sim.chains_init(x0)
        tr = torch.empty((37, C), dtype=torch.int64, device="cuda:0")
        po = torch.empty(C, dtype=torch.float64, device="cuda:0")
        sim.metropolis(37, seed=77, trace=tr, p_out=po)
        xo = torch.empty(C, dtype=torch.int64, device="cuda:0")
        po2 = torch.empty(C, dtype=torch.float64, device="cuda:0")
        sim.metropolis(35, seed=78, step0=37, x_out=xo, p_out=po2)
        res[look] = (tr.cpu(), po.cpu(), xo.cpu(), po2.cpu())
    for a, b in zip(res[1], res[2]):
        assert torch.equal(a, b)
    moved = (res[2][0][-1] != x0.cpu()).sum().item()
    assert moved > C // 4          # the chains do move
    sim.close()
