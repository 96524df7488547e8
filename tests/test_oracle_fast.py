"""Pins for the C restatement of the oracle (oracle/c/chform_oracle.c through
oracle/fast.py): every term's tableau, phases and omega bit-exact against the Python
oracle; exact amplitude and overlap sums equal to the Python oracle's exact sums and to
the dense state vector; the hidden shift exactly; the same integers for every thread
count."""
import random

import numpy as np
import pytest

from oracle import decomp, dense, exact, fast
from oracle import estimators as E
from paper_1808_00128_gb300 import workloads
from tests._circuits import rand_clifford


def _compare_terms(n, ops, chi, mode, seed, alphas, ccz_mode="proj"):
    prep = fast.Prepared(n, ops, chi, mode, seed, ccz_mode)
    terms, _, chs = decomp.build_decomposition(n, ops, chi=chi, mode=mode, seed=seed, ccz_mode=ccz_mode,
                                               alphas=alphas)
    ed = exact.ExactDecomposition(n, ops, chi, mode, ccz_mode)
    for a, t, ch in zip(alphas, terms, chs):
        F, G, M, gam, v, s, zero, k, h, Ma, es = prep.term(a)
        assert (F, G, M, gam, v, s, zero) == (t.F, t.G, t.M, t.gamma, t.v, t.s, t.zero), (n, a)
        if not zero:
            assert (k, h) == (t.k % 8, t.h), (n, a)
        assert Ma % 8 == ed.parts(ch)[2]
    return prep, terms, chs, ed


def test_benchmark_workloads_term_by_term():
    for cfg in (workloads.config_tiny(), workloads.config_mid(), workloads.config_qaoa()):
        alphas = list(range(cfg["chi"])) if cfg["chi"] <= 64 else [0, 1, 4097, cfg["chi"] // 2, cfg["chi"] - 1]
        _compare_terms(cfg["n"], cfg["ops"], cfg["chi"], cfg["mode"], cfg["seed"], alphas)


@pytest.mark.parametrize("n", [1, 2, 5, 33, 63, 64])
def test_random_circuits_with_projectors_term_by_term(n):
    rng = random.Random(300 + n)
    ops = rand_clifford(n, 4 * n + 20, rng)
    ops.insert(rng.randrange(len(ops) + 1), ("T", rng.randrange(n)))
    ops.insert(rng.randrange(len(ops) + 1), ("RZ", rng.randrange(n), -0.7))
    if n >= 3:
        ops.insert(rng.randrange(len(ops) + 1), ("CCZ", *rng.sample(range(n), 3)))
    _compare_terms(n, ops, 40, "sparsify", 9, list(range(0, 40, 3)))
    if n >= 3:
        _compare_terms(n, ops, 40, "sparsify", 9, list(range(0, 40, 7)), ccz_mode="sum8")


def test_exact_sums_equal_python_exact_and_dense():
    cfg = workloads.config_tiny()
    n, ops, chi = cfg["n"], cfg["ops"], cfg["chi"]
    prep, terms, chs, ed = _compare_terms(n, ops, chi, "exact", 0, list(range(chi)))
    coefs = [decomp.coefficient(decomp.lower(ops)[1], ch, "exact", chi) for ch in chs]
    psi = dense.run(n, ops)
    xs = list(range(0, 1 << n, 7))
    As = [E.draw_A(n, 4, l) for l in range(4)]
    amps, ovs = prep.sums(xs, As)
    for x, a in zip(xs, amps):
        assert abs(fast.to_complex(a) - exact.to_complex(ed.amplitude(terms, chs, x))) < 1e-15
        assert abs(fast.to_complex(a) - psi[x]) < 1e-13
    for A, o in zip(As, ovs):
        want = ed.overlap_A(terms, chs, A)
        assert abs(fast.to_complex(o) - exact.to_complex(want)) < 1e-15
        assert abs(fast.eta_of(o, n) - E.eta(terms, coefs, A)) < 1e-12


def test_hidden_shift_exact_and_thread_count_independent():
    """Integer coefficients (exact CCZ form): <s|psi> = 1 and <x|psi> = 0 exactly, and
    the integer sums do not depend on how the terms are split over threads."""
    n = 8
    ops, s = workloads.hidden_shift_circuit(n, 4, seed=12)
    prep = fast.Prepared(n, ops, 16, "exact")
    xs = list(range(1 << n))
    r1, _ = prep.sums(xs, threads=1)
    r5, _ = prep.sums(xs, threads=5)
    assert r1 == r5
    for x, a in zip(xs, r1):
        assert fast.to_complex(a) == (1.0 if x == s else 0.0)


def test_sparsified_sums_against_python_oracle():
    n = 12
    ops = workloads.random_clifford_t(n, 150, 7, seed=77) + [("RZ", 3, 0.45)]
    chi, seed = 60, 4
    prep, terms, chs, ed = _compare_terms(n, ops, chi, "sparsify", seed, list(range(chi)))
    coefs = [decomp.coefficient(decomp.lower(ops)[1], ch, "sparsify", chi) for ch in chs]
    xs = [t.sample(1234567 * (i + 1)) for i, t in enumerate(terms[:20])] + [5, 77, 4095]
    As = [E.draw_A(n, 8, l) for l in range(3)]
    amps, ovs = prep.sums(xs, As, threads=3)
    for x, a in zip(xs, amps):
        want = E.amplitude(terms, coefs, x)
        assert abs(fast.to_complex(a) - want) <= 1e-13 * max(1.0, abs(want))
    for A, o in zip(As, ovs):
        assert abs(fast.to_complex(o) - E.overlap_A(terms, coefs, A)) < 1e-13
