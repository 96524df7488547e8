"""Host logic of the benchmark (no GPU): the algorithmic work models behind the
roofline fractions, the step's unit count, the autocorrelation time of the sampler
study, and the command-line defaults the benchmark contract fixes."""
import sys

import numpy as np

import bench
from paper_1808_00128_gb300 import lrstab


def test_clifford_op_model_per_gate():
    n = 3
    # H on an untouched qubit acts on |0>: constant part only; every later H pays the
    # row pass 30 n + 40; CX 12, S 4, CZ 4, Z 2 (32-bit op equivalents)
    low = lrstab.lower_circuit(n, [("H", 0), ("H", 0), ("CX", 0, 1), ("S", 1), ("H", 1), ("CZ", 1, 2), ("Z", 2)])
    want = 40 + (30 * n + 40) + 12 + 4 + (30 * n + 40) + 4 + 2
    assert bench.clifford_ops_per_term(n, low) == want


def test_clifford_op_model_weights_slot_choices():
    # a T slot: K_0 = I (no gates), K_1 = a diagonal Clifford; its cost is the
    # choice-weighted mean of the K lists' costs
    n = 2
    low = lrstab.lower_circuit(n, [("H", 0), ("T", 0)])
    s = low.slots[0]
    nc = int(s["n_choices"])
    w = np.hypot(s["c_re"][:nc], s["c_im"][:nc])
    w = w / w.sum()
    inv = {v: k for k, v in lrstab.OP.items()}
    per_choice = []
    for j in range(nc):
        sub = low.kgates[s["k_off"][j]: s["k_off"][j] + s["k_len"][j]]
        per_choice.append(sum(bench.GATE_OPS.get(inv[int(k["op"])], 0) for k in sub))
    assert abs(bench.clifford_ops_per_term(n, low) - (40 + float(np.dot(w, per_choice)))) < 1e-9


def test_norm_op_model_by_route():
    n = 40
    vw = np.array([40, 38, 20])
    got = bench.norm_ops_per_unit(n, vw, 12)
    m = n - vw
    assert got[0] == 8 * n + 4 * 40 ** 2                      # no constraint to fold
    assert got[1] == 8 * n + 5 * 2 * n + 4 * 38 ** 2          # two folded constraints
    assert got[2] == 8 * n * n + 4 * 20 ** 2                  # 20 > 12: K path
    assert np.all(bench.norm_ops_per_unit(n, vw, -1) == 8 * n * n + 4 * vw ** 2)
    assert m[2] > 12


def test_units_and_launches_per_step():
    chi = 1 << 20
    s = bench.SHAPES["qaoa"]
    assert bench.units_per_step(chi, s["B"], s["C"], s["T"]) == chi * (4096 + 256 * 65)
    # init, apply, amplitude (2), norm (4), chain starts, chains_init (3), Metropolis:
    # set + first + 4 graphs of 16 steps (33 launches each) + out
    assert bench.launches_per_step(64) == 1 + 1 + 2 + 4 + 1 + 3 + 2 + 4 * 33 + 1
    assert bench.launches_per_step(18) == 1 + 1 + 2 + 4 + 1 + 3 + 2 + 33 + 4 + 1
    # two steps per pass: 8 passes (16 launches) + advance per graph; 3 leftover steps
    # take one pass and one single step
    assert bench.launches_per_step(64, 2) == 1 + 1 + 2 + 4 + 1 + 3 + 2 + 4 * 17 + 1
    assert bench.launches_per_step(19, 2) == 1 + 1 + 2 + 4 + 1 + 3 + 2 + 17 + 4 + 1


def test_formula_and_kernel_counts():
    """The hot-path table's formulas count every H at 30 n + 40, every (x, term) at
    10 |x| + 30 and every (A, term) at 8 n^2 + 4 |v|^2; the kernel counts are lower."""
    n = 4
    low = lrstab.lower_circuit(n, [("H", 0), ("H", 1), ("CX", 0, 1)])
    assert bench.clifford_ops_per_term(n, low, formula=True) == 2 * (30 * n + 40) + 12
    assert bench.clifford_ops_per_term(n, low) == 2 * 40 + 12
    assert bench.amplitude_ops_per_unit(50, 25.0, formula=True) == 280.0
    assert bench.amplitude_ops_per_unit(50, 25.0) == 8 * 13 + 16
    assert bench.metropolis_bytes(2, 3, 5, 10) == 5 * (2 * 3 * 24 + 2 * 160)
    # two steps per pass: states read once per pass, written back with probability
    # 1 - (1 - 1/2)^2, rows of both proposals; the fifth step is a single step
    assert bench.metropolis_bytes(2, 3, 5, 10, lookahead=2) == 2 * (2 * 3 * 28 + 2 * 2 * 160) + (2 * 3 * 24 + 2 * 160)


def test_traffic_is_dropped_when_the_kernel_changes(monkeypatch):
    sha = bench.source_sha16("bench.py")
    monkeypatch.setitem(bench.TRAFFIC, "norm_estimate",
                        {"bytes_per_unit": 2.0, "source": "bench.py", "sha16": sha, "profile": "p.md"})
    assert bench.traffic_for("norm_estimate", 10) == (20.0, "p.md")
    monkeypatch.setitem(bench.TRAFFIC, "norm_estimate",
                        {"bytes_per_unit": 2.0, "source": "bench.py", "sha16": "0" * 16, "profile": "p.md"})
    t, src = bench.traffic_for("norm_estimate", 10)
    assert t is None and "changed" in src
    assert bench.traffic_for("amplitude", 10) == (None, None)


def test_oracle_step_time_model():
    rates = {"t_build": 1e-3, "t_amp": 1e-6, "t_inner": 1e-4, "parallel": 4.0}
    s = dict(B=10, L=3, C=2, T=4)
    want = 8 * (1e-3 + (10 + 2 * 5) * 1e-6 + 3 * 1e-4) / 4.0
    assert abs(bench.oracle_step_seconds(8, s, rates) - want) < 1e-15


def test_tau_int_white_noise_and_ar1():
    rng = np.random.default_rng(0)
    white = rng.standard_normal((4000, 64))
    assert abs(bench.tau_int(white) - 1.0) < 0.15
    # AR(1) with coefficient r: tau = (1 + r) / (1 - r)
    r = 0.8
    x = np.zeros((4000, 64))
    e = rng.standard_normal((4000, 64))
    for t in range(1, 4000):
        x[t] = r * x[t - 1] + e[t]
    assert abs(bench.tau_int(x) - (1 + r) / (1 - r)) < 1.0
    assert bench.tau_int(np.ones((10, 3))) == 1.0


def test_command_line_defaults(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.impl) == (1, "lrstab")
    assert a.warmup >= 3 and a.steps >= 1
