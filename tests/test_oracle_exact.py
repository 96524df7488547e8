"""Pins for the oracle's exact Z[zeta8] chi-sums (oracle/exact.py): closed forms of
the accumulator, the dense state vector, the FP64 oracle, and identities that hold
exactly (the hidden shift's zero amplitudes, unit norm of integer-coefficient
decompositions, the exhaustive average of Lemma (Norm Estimation))."""
import cmath
import math
import random
from decimal import Decimal

import numpy as np
import pytest

from oracle import decomp, dense, exact
from oracle import estimators as E
from paper_1808_00128_gb300 import workloads


def test_z8_accumulator_closed_forms():
    """zeta^K 2^{-e/2} for every K mod 8 and e in 0..9 (odd e through the sqrt2
    identity), and exact cancellation of opposite terms."""
    for K in range(-8, 16):
        for e in range(10):
            acc = exact.Z8Sum(S=16)
            acc.add(K, e)
            want = cmath.exp(1j * math.pi * (K % 8) / 4) * 2.0 ** (-e / 2)
            got = exact.to_complex(acc.decimal())
            assert abs(got - want) < 1e-15, (K, e)
            acc.add(K + 4, e)             # zeta^4 = -1
            assert acc.is_zero()


def test_slot_factors_of_the_lowerings():
    """T, RZ (both signs) and both CCZ forms factor as r g zeta^m; a slot with a
    phase that is not a multiple of pi/4 does not."""
    for op in (("T", 0), ("RZ", 0, 0.3), ("RZ", 0, -0.7), ("CCZ_SUM8", 0, 1, 2), ("CCZ_PROJ", 0, 1, 2)):
        dec = decomp.gate_decomposition(op)
        ch, g = exact.slot_factors(dec)
        for (c, _), (r, m) in zip(dec, ch):
            assert abs(c - r * g * cmath.exp(1j * math.pi * m / 4)) < 1e-15
    assert exact.slot_factors([(1.0, []), (cmath.exp(0.3j), [])]) is None


def _case(n, ops, chi, mode, seed=0, ccz_mode="proj"):
    terms, coefs, chs = decomp.build_decomposition(n, ops, chi=chi, mode=mode, seed=seed, ccz_mode=ccz_mode)
    ex = exact.ExactDecomposition(n, ops, chi, mode, ccz_mode)
    return terms, coefs, chs, ex


@pytest.mark.parametrize("mode", ["exact", "sparsify"])
def test_exact_amplitudes_equal_fp64_oracle_and_dense(mode):
    rng = random.Random(7)
    for trial in range(6):
        n = rng.randrange(3, 9)
        ops = workloads.random_clifford_t(n, 40, 3, seed=100 + trial)
        ops += [("RZ", rng.randrange(n), rng.uniform(-1, 1)), ("CCZ", 0, 1, 2)]
        ccz_mode = "sum8" if trial % 2 else "proj"
        chi = decomp.exact_chi(decomp.lower(ops, ccz_mode)[1]) if mode == "exact" else 24
        terms, coefs, chs, ex = _case(n, ops, chi, mode, seed=trial, ccz_mode=ccz_mode)
        if mode == "exact":
            psi = dense.run(n, ops)
        for x in range(1 << n):
            got = exact.to_complex(ex.amplitude(terms, chs, x))
            want = E.amplitude(terms, coefs, x)
            assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (trial, x)
            if mode == "exact":
                assert abs(got - psi[x]) <= 1e-13


def test_hidden_shift_is_exact():
    """Sec. 2.4.2: the hidden-shift circuit maps |0^n> to |s>.  With the exact
    projector form of CCZ (integer coefficients 1, -2) every chi-sum is exact:
    <s|psi> = 1 and <x|psi> = 0 with no rounding at all, where the FP64 sum leaves
    residues."""
    n = 8
    ops, s = workloads.hidden_shift_circuit(n, 4, seed=12)
    chi = 16
    terms, coefs, chs, ex = _case(n, ops, chi, "exact")
    one = ex.amplitude(terms, chs, s)
    assert one == (Decimal(1), Decimal(0))
    for x in range(1 << n):
        if x != s:
            assert ex.amplitude(terms, chs, x) == (Decimal(0), Decimal(0))


def test_unit_norm_exact_decomposition():
    """sum_x |<x|psi>|^2 = 1 for the exact T decomposition (magnitudes are FP64 values
    of sqrt2 sin(pi/8), hence 1e-15) and exactly for integer CCZ coefficients."""
    n = 6
    ops = workloads.random_clifford_t(n, 60, 4, seed=5)
    terms, coefs, chs, ex = _case(n, ops, 16, "exact")
    tot = sum(exact.abs_decimal(ex.amplitude(terms, chs, x)) ** 2 for x in range(1 << n))
    assert abs(float(tot) - 1.0) < 1e-14
    ops = [("H", q) for q in range(n)] + [("CCZ", 0, 1, 2), ("CZ", 2, 3), ("CCZ", 3, 4, 5), ("H", 1), ("H", 4)]
    terms, coefs, chs, ex = _case(n, ops, 4, "exact")
    tot = sum(exact.abs_decimal(ex.amplitude(terms, chs, x)) ** 2 for x in range(1 << n))
    assert abs(tot - 1) < Decimal(10) ** -50


def test_exact_eta_equals_fp64_and_exhaustive_average():
    """Exact eta_A agrees with the FP64 oracle; with integer coefficients the average
    over all of M_n equals ||psi||^2 exactly (Lemma (Norm Estimation))."""
    n = 3
    ops = [("H", 0), ("H", 1), ("H", 2), ("CCZ", 0, 1, 2), ("H", 0), ("S", 1), ("CCZ", 0, 1, 2), ("CX", 1, 2)]
    terms, coefs, chs, ex = _case(n, ops, 4, "exact")
    norm2 = sum(exact.abs_decimal(ex.amplitude(terms, chs, x)) ** 2 for x in range(1 << n))
    tot, cnt = Decimal(0), 0
    for A in E.all_equatorial(n):
        e = ex.eta(terms, chs, A)
        assert abs(float(e) - E.eta(terms, coefs, A)) < 1e-12
        tot += e
        cnt += 1
    assert abs(tot / cnt - norm2) < Decimal(10) ** -45
    # sparsified T/RZ decompositions at n = 10: exact eta against the FP64 oracle
    n = 10
    ops = workloads.random_clifford_t(n, 120, 6, seed=9) + [("RZ", 3, 0.4)]
    terms, coefs, chs, ex = _case(n, ops, 40, "sparsify", seed=2)
    for l in range(6):
        A = E.draw_A(n, 11, l)
        assert abs(float(ex.eta(terms, chs, A)) - E.eta(terms, coefs, A)) < 1e-12 * max(1.0, E.eta(terms, coefs, A))
