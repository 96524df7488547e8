"""Full-size oracle sums through the plain C restatement of the oracle (test
infrastructure only; oracle/c/chform_oracle.c).

The Python oracle builds one term in tens of milliseconds at n = 50; the benchmark's
decompositions hold 2^16..2^20 terms.  The C file restates the same CH-form rules,
decomposition choices, amplitude and inner-product formulas and exact Z[zeta8]
accumulation (the readings of oracle/chform.py, oracle/decomp.py,
oracle/estimators.py and oracle/exact.py), builds every term on the fly on all host
threads and returns exact integer sums; this module prepares the circuit from the
Python oracle's own lowering and slot factors and converts the sums once, in 60-digit
decimal arithmetic.  The tests pin it against the Python oracle term by term.

Supported decompositions: sparsify mode, and exact mode when the magnitudes of each
slot's choices differ by powers of sqrt2 (T, CCZ in both forms; RZ in exact mode only
for angles where that holds).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from decimal import Decimal, localcontext

import numpy as np

from . import exact
from .decomp import l1_norm, lower

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "c", "chform_oracle.c")
LIB = os.path.join(_HERE, "c", "libchform_oracle.so")
EX_S = 100
OPS = dict(H=0, S=1, SDG=2, Z=3, X=4, CX=5, CZ=6, P0=7, P1=8, SLOT=9)
_PREC = 60


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, plain C, pthreads) next to its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O3", "-std=gnu11", "-shared", "-fPIC", "-pthread", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"C oracle build failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        p, i64, i32, u64 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64
        L.oracle_sums.argtypes = [i32, i64, p, i64, p, p, p, p, p, p, p, p, i32, u64, i64, i64, p, i64, p, i64,
                                  i32, p]
        L.oracle_sums.restype = C.c_int
        L.oracle_term.argtypes = [i32, i64, p, i64, p, p, p, p, p, p, p, p, i32, u64, i64, p, p, p]
        L.oracle_term.restype = C.c_int
        _lib = L
    return _lib


def _gate_row(g):
    name = g[0]
    if name == "SLOT":
        return [OPS["SLOT"], 0, g[1]]
    if name in ("CX", "CZ"):
        return [OPS[name], g[1], g[2]]
    return [OPS[name], g[1], 0]


class Prepared:
    """A lowered decomposition in the C oracle's arrays, with the factor common to
    every coefficient: b_alpha = common * zeta^{M_alpha} * 2^{-eshift_alpha / 2}."""

    def __init__(self, n: int, ops, chi_total: int, mode: str, seed: int = 0, ccz_mode: str = "proj"):
        gates, slots = lower(ops, ccz_mode)
        factors = exact.decomposition_factors(slots)
        if factors is None:
            raise ValueError("slot coefficients do not factor as r g zeta^m")
        self.n, self.chi_total, self.mode, self.seed = n, chi_total, mode, seed
        self.gates = np.array([_gate_row(g) for g in gates], np.int32).reshape(-1, 3)
        ns = max(1, len(slots))
        self.n_choices = np.zeros(ns, np.int32)
        self.k_off = np.zeros((ns, 8), np.int32)
        self.k_len = np.zeros((ns, 8), np.int32)
        self.phase_m = np.zeros((ns, 8), np.int32)
        self.e_shift = np.zeros((ns, 8), np.int32)
        self.cdf = np.zeros((ns, 8), np.float64)
        self.nonzero = np.zeros((ns, 8), np.int32)
        kg = []
        common_mag = 1.0
        for p, (dec, (ch, _g)) in enumerate(zip(slots, factors)):
            self.n_choices[p] = len(dec)
            norm = sum(abs(c) for c, _ in dec)
            acc = 0.0
            rs = [r for r, _ in ch if r > 0]
            r_ref = min(rs)
            common_mag *= r_ref
            for j, ((c, K), (r, m)) in enumerate(zip(dec, ch)):
                self.k_off[p, j] = len(kg)
                self.k_len[p, j] = len(K)
                kg += [_gate_row(k) for k in K]
                self.phase_m[p, j] = m
                self.nonzero[p, j] = 1 if c != 0 else 0
                if c != 0:
                    acc += abs(c) / norm
                self.cdf[p, j] = acc
                if mode == "exact" and r > 0:
                    ratio = r / r_ref
                    k2 = round(2 * math.log2(ratio))
                    if abs(ratio - 2.0 ** (k2 / 2)) > 1e-12 * ratio:
                        raise ValueError("exact-mode magnitudes of a slot differ by other than powers of sqrt2")
                    self.e_shift[p, j] = -k2
        self.kgates = np.array(kg if kg else [[0, 0, 0]], np.int32).reshape(-1, 3)
        self.n_slots = len(slots)
        G = exact.common_phase(factors)
        mag = l1_norm(slots) / chi_total if mode == "sparsify" else common_mag
        self.common = (Decimal(mag) * Decimal(G.real), Decimal(mag) * Decimal(G.imag))

    def _args(self):
        return [self.n, len(self.gates), self.gates.ctypes.data, self.n_slots, self.n_choices.ctypes.data,
                self.k_off.ctypes.data, self.k_len.ctypes.data, self.kgates.ctypes.data, self.phase_m.ctypes.data,
                self.e_shift.ctypes.data, self.cdf.ctypes.data, self.nonzero.ctypes.data,
                0 if self.mode == "exact" else 1, self.seed & (2 ** 64 - 1)]

    def term(self, alpha: int):
        """(F, G, M, gamma, v, s, zero, k mod 8, h, M_alpha, eshift) of term alpha."""
        n = self.n
        rows = np.zeros(3 * n, np.uint64)
        gam = np.zeros(n, np.int32)
        sc = np.zeros(7, np.int64)
        rc = lib().oracle_term(*self._args(), alpha, rows.ctypes.data, gam.ctypes.data, sc.ctypes.data)
        if rc:
            raise RuntimeError("oracle_term failed")
        return ([int(v) for v in rows[:n]], [int(v) for v in rows[n:2 * n]], [int(v) for v in rows[2 * n:]],
                [int(g) for g in gam], int(sc[0]) & (2 ** 64 - 1), int(sc[1]) & (2 ** 64 - 1), bool(sc[2]),
                int(sc[3]), int(sc[4]), int(sc[5]), int(sc[6]))

    def sums(self, xs=(), As=(), alpha0: int = 0, count: int | None = None, threads: int | None = None):
        """Exact <x|psi> for each x and <phi_A|psi> for each A (integer matrices) over the
        terms [alpha0, alpha0 + count), as (Re, Im) Decimal pairs."""
        count = self.chi_total - alpha0 if count is None else count
        threads = threads or max(1, os.cpu_count() or 1)
        x = np.ascontiguousarray(np.asarray(list(xs), dtype=np.uint64).reshape(-1))
        n = self.n
        A = np.ascontiguousarray(np.asarray(list(As), dtype=np.int8).reshape(-1, n, n)) if len(As) else \
            np.zeros((0, n, n), np.int8)
        rows = len(x) + len(A)
        out = np.zeros(8 * max(rows, 1), np.int64)
        rc = lib().oracle_sums(*self._args(), alpha0, count, x.ctypes.data if len(x) else None, len(x),
                               A.ctypes.data if len(A) else None, len(A), threads, out.ctypes.data)
        if rc:
            raise RuntimeError("oracle_sums failed")
        res = []
        with localcontext() as ctx:
            ctx.prec = _PREC
            r2 = Decimal(2).sqrt()
            sc = Decimal(2) ** (-EX_S)
            for r in range(rows):
                c = []
                for j in range(4):
                    lo = int(out[8 * r + 2 * j]) & (2 ** 64 - 1)
                    hi = int(out[8 * r + 2 * j + 1])
                    c.append(Decimal(lo + (hi << 64)))
                re = (c[0] + (c[1] - c[3]) / r2) * sc
                im = (c[2] + (c[1] + c[3]) / r2) * sc
                cr, ci = self.common
                res.append((re * cr - im * ci, re * ci + im * cr))
        return res[:len(x)], res[len(x):]


def to_complex(z) -> complex:
    return complex(float(z[0]), float(z[1]))


def eta_of(z, n: int) -> float:
    """2^n |z|^2 for an overlap given as a Decimal pair."""
    with localcontext() as ctx:
        ctx.prec = _PREC
        return float((Decimal(2) ** n) * (z[0] * z[0] + z[1] * z[1]))
