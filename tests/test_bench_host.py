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


def test_units_per_step():
    chi = 1 << 16
    assert bench.units_per_step(chi) == chi * (bench.B_X + bench.C_CH * (bench.T_MC + 1))


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
