"""Bit-exact parity of the CUDA term pipeline (init_terms + apply_clifford)
with the oracle CH-form simulator: tableaux, phase vectors, v, s and the exact
omega (Z8 phase, power of sqrt2, zero flag)."""
import random

import numpy as np
import pytest
import torch

from oracle import decomp
from oracle.chform import CHForm, run_gates
from paper_1808_00128_gb300 import lrstab, workloads
from tests._gpu import compare_term, oracle_terms, require_cuda

pytestmark = pytest.mark.gpu


def _run(n, ops, chi, mode, seed=0, ccz_mode="proj", alpha0=0, chi_total=None):
    low = lrstab.lower_circuit(n, ops, ccz_mode)
    sim = lrstab.Simulator(n, 0)
    sim.init_terms(low, chi, mode=mode, seed=seed, alpha0=alpha0, chi_total=chi_total)
    sim.apply_clifford(low.gates)
    return sim, low


def test_tiny_config_all_terms_bit_exact():
    require_cuda()
    cfg = workloads.config_tiny()
    n, ops = cfg["n"], cfg["ops"]
    sim, low = _run(n, ops, cfg["chi"], "exact")
    ex = sim.export_terms()
    terms, coefs, chs = oracle_terms(n, ops, cfg["chi"], "exact")
    for a in range(cfg["chi"]):
        compare_term(ex, a, terms[a], f"term {a}")
        assert list(ex["choice"][a][: len(chs[a])]) == chs[a]
        b = complex(ex["coef"][a][0], ex["coef"][a][1])
        assert abs(b - coefs[a]) <= 1e-6 * abs(coefs[a])
    sim.close()


def _random_circuit(n, n_gates, n_t, n_ccz, rng):
    ops = []
    for _ in range(n_gates):
        k = rng.randrange(5)
        if k == 0:
            ops.append(("H", rng.randrange(n)))
        elif k == 1:
            ops.append((rng.choice(["S", "SDG", "Z"]), rng.randrange(n)))
        elif n > 1:
            a, b = rng.sample(range(n), 2)
            ops.append(("CX" if k < 4 else "CZ", a, b))
    for _ in range(n_t):
        ops.insert(rng.randrange(len(ops) + 1), ("T", rng.randrange(n)))
    for _ in range(n_ccz):
        ops.insert(rng.randrange(len(ops) + 1), ("CCZ", *rng.sample(range(n), 3)))
    return ops


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 39, 40, 41, 48, 49, 50, 56, 57, 62, 63, 64])
def test_edge_widths_bit_exact(n):
    """Exact decompositions with T and projector-form CCZ at edge register widths."""
    require_cuda()
    rng = random.Random(1000 + n)
    n_ccz = 2 if n >= 3 else 0
    ops = _random_circuit(n, 6 * n + 20, 3, n_ccz, rng)
    chi = 2 ** (3 + n_ccz)
    sim, low = _run(n, ops, chi, "exact")
    ex = sim.export_terms()
    terms, _, _ = oracle_terms(n, ops, chi, "exact", parallel=True)
    for a in range(chi):
        compare_term(ex, a, terms[a], f"n={n} term {a}")
    sim.close()


def test_gate_list_longer_than_one_launch():
    """More gates than one launch carries (7680): the list is split over launches."""
    require_cuda()
    rng = random.Random(77)
    n = 9
    ops = _random_circuit(n, 16000, 2, 1, rng)
    chi = 2 ** 3
    sim, low = _run(n, ops, chi, "exact")
    assert len(low.gates) > 2 * 7680
    ex = sim.export_terms()
    terms, _, _ = oracle_terms(n, ops, chi, "exact", parallel=True)
    for a in range(chi):
        compare_term(ex, a, terms[a], f"term {a}")
    sim.close()


def test_all_hadamard_v_full():
    """|v| = 64: H on every qubit of a 64-qubit register."""
    require_cuda()
    n = 64
    ops = [("H", q) for q in range(n)] + [("CZ", q, (q + 1) % n) for q in range(0, n, 2)] + [("T", 5)]
    sim, low = _run(n, ops, 2, "exact")
    ex = sim.export_terms()
    terms, _, _ = oracle_terms(n, ops, 2, "exact")
    for a in range(2):
        compare_term(ex, a, terms[a])
        assert int(ex["v"][a]) == (1 << 64) - 1
    sim.close()


def test_projectors_and_raw_gates():
    """Raw gate lists with P0/P1 projectors (terms may vanish) through apply_clifford."""
    require_cuda()
    rng = random.Random(7)
    for trial in range(12):
        n = rng.randrange(2, 12)
        gates = []
        for _ in range(60):
            k = rng.randrange(7)
            q = rng.randrange(n)
            if k == 0:
                gates.append(("H", q))
            elif k == 1:
                gates.append(("S", q))
            elif k == 2:
                gates.append(("SDG", q))
            elif k == 3:
                gates.append((rng.choice(["P0", "P1"]), q))
            else:
                r = rng.choice([i for i in range(n) if i != q])
                gates.append(("CX" if k < 6 else "CZ", q, r))
        sim = lrstab.Simulator(n, 0)
        empty = lrstab.lower_circuit(n, [])
        sim.init_terms(empty, 1, mode="exact")
        sim.apply_clifford(lrstab.gates_array(gates))
        ex = sim.export_terms()
        ch = run_gates(n, gates)
        compare_term(ex, 0, ch, f"trial {trial}")
        sim.close()


def test_mid_config_slice_choices_and_terms():
    """n=40 circuit (2000 Cliffords + 24 T), sparsified chi_total = 2^16; a ragged
    slice of 300 terms: every choice and coefficient, and sampled terms bit-exact."""
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, chi_total = cfg["n"], cfg["ops"], cfg["chi"]
    alpha0, chi = 12345, 300
    sim, low = _run(n, ops, chi, "sparsify", seed=77, alpha0=alpha0, chi_total=chi_total)
    ex = sim.export_terms()
    gates, slots = decomp.lower(ops)
    l1 = decomp.l1_norm(slots)
    for i in range(chi):
        want = decomp.choices_sparsify(slots, alpha0 + i, 77)
        assert list(ex["choice"][i][: len(slots)]) == want, f"choices of term {alpha0 + i}"
        b = complex(ex["coef"][i][0], ex["coef"][i][1])
        bw = decomp.coefficient(slots, want, "sparsify", chi_total)
        assert abs(b - bw) <= 1e-6 * abs(bw)
    pick = [0, 1, 150, 299]
    terms, _, _ = oracle_terms(n, ops, chi_total, "sparsify", seed=77,
                               alphas=[alpha0 + i for i in pick], parallel=True)
    for i, t in zip(pick, terms):
        compare_term(ex, i, t, f"term {alpha0 + i}")
    assert l1 > 1
    sim.close()


def test_mid_config_full_size_sampled_terms():
    """The full chi = 2^16 launch the benchmark times; 8 sampled terms bit-exact."""
    require_cuda()
    cfg = workloads.config_mid()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    sim, low = _run(n, ops, chi, "sparsify", seed=cfg.get("seed", 1))
    rng = random.Random(3)
    pick = sorted(rng.sample(range(chi), 8)) + [chi - 1]
    terms, _, _ = oracle_terms(n, ops, chi, "sparsify", seed=cfg.get("seed", 1), alphas=pick,
                               parallel=True)
    for a, t in zip(pick, terms):
        ex = sim.export_terms(a, 1)
        compare_term(ex, 0, t, f"term {a}")
    sim.close()


def test_qaoa_full_size_sampled_terms():
    """n=50 QAOA circuit sparsified to chi = 2^20 (the 24-bit high-word tableau layout);
    sampled terms bit-exact."""
    require_cuda()
    cfg = workloads.config_qaoa()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    sim, low = _run(n, ops, chi, "sparsify", seed=cfg["seed"])
    rng = random.Random(5)
    pick = sorted(rng.sample(range(chi), 5)) + [chi - 1]
    terms, _, _ = oracle_terms(n, ops, chi, "sparsify", seed=cfg["seed"], alphas=pick, parallel=True)
    for a, t in zip(pick, terms):
        compare_term(sim.export_terms(a, 1), 0, t, f"term {a}")
    sim.close()


def test_hidden_shift_full_size_sampled_terms():
    require_cuda()
    cfg = workloads.config_hidden_shift()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    sim, low = _run(n, ops, chi, "exact")
    pick = [0, 1, 2 ** 15 + 3, chi - 1]
    terms, _, _ = oracle_terms(n, ops, chi, "exact", alphas=pick, parallel=True)
    for a, t in zip(pick, terms):
        compare_term(sim.export_terms(a, 1), 0, t, f"term {a}")
    sim.close()


def test_sample_terms_matches_oracle_sampler():
    require_cuda()
    from oracle import rng as orng
    cfg = workloads.config_tiny()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    sim, low = _run(n, ops, chi, "exact")
    count = 200
    alpha = torch.empty(count, dtype=torch.int64, device="cuda:0")
    x = sim.sample_terms(count, seed=9, alpha=alpha)
    x, alpha = x.cpu().numpy(), alpha.cpu().numpy()
    terms, _, _ = oracle_terms(n, ops, chi, "exact")
    for i in range(count):
        a = (orng.rand64(9, i, 0) * chi) >> 64
        assert alpha[i] == a
        flips = orng.rand64(9, i, 1)
        assert int(x[i]) == terms[a].sample(flips)
        assert abs(terms[a].amplitude(int(x[i]))) > 0
    sim.close()


@pytest.mark.parametrize("lanes", [1, 2, 4])
@pytest.mark.parametrize("n", [49, 50, 57, 63, 64])
def test_lane_split_bit_exact(n, lanes):
    """The 64-bit-row kernel with 1, 2 or 4 lanes per term (each lane owns the rows
    p = part mod lanes): exact decompositions with T and projector-form CCZ, every
    term bit-exact against the oracle."""
    require_cuda()
    rng = random.Random(2000 + n)
    ops = _random_circuit(n, 5 * n, 3, 2, rng)
    chi = 2 ** 5
    low = lrstab.lower_circuit(n, ops)
    sim = lrstab.Simulator(n, 0)
    sim.set_tuning("apply_lanes", lanes)
    sim.init_terms(low, chi, mode="exact")
    sim.apply_clifford(low.gates)
    ex = sim.export_terms()
    terms, _, _ = oracle_terms(n, ops, chi, "exact", parallel=True)
    for a in range(chi):
        compare_term(ex, a, terms[a], f"n={n} lanes={lanes} term {a}")
    sim.close()


def test_lane_split_qaoa_n50_identical_terms():
    """The n = 50 QAOA circuit (gamma 0.3, beta 0.2) on 2^14 sparsified terms: 1, 2 and 4
    lanes per term give the same tableaux, phases and omega for every term, and a
    64-term sample equals the oracle bit for bit."""
    require_cuda()
    cfg = workloads.config_qaoa()
    n, ops, seed = cfg["n"], cfg["ops"], cfg["seed"]
    chi = 1 << 14
    low = lrstab.lower_circuit(n, ops)
    out = {}
    for lanes in (1, 2, 4):
        sim = lrstab.Simulator(n, 0)
        sim.set_tuning("apply_lanes", lanes)
        sim.init_terms(low, chi, mode="sparsify", seed=seed, chi_total=cfg["chi"])
        sim.apply_clifford(low.gates)
        out[lanes] = sim.export_terms()
        sim.close()
    for k in out[1]:
        assert np.array_equal(out[1][k], out[2][k]), k
        assert np.array_equal(out[1][k], out[4][k]), k
    alphas = list(range(0, chi, chi // 64))
    terms, _, _ = oracle_terms(n, ops, cfg["chi"], "sparsify", seed=seed, alphas=alphas, parallel=True)
    for i, a in enumerate(alphas):
        compare_term(out[2], a, terms[i], f"term {a}")
