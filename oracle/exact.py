"""Exact chi-sums in Z[zeta8] (oracle; test infrastructure only).

Every per-term value of the method is an exact phase times a power of sqrt2 times
the term's coefficient:
  * amplitudes (Eqs. (amplitude), (amplitude1)):
        b_alpha <x|phi_alpha> = b_alpha zeta^{k + 2 mu + 4 sign} 2^{-(|v| + h)/2}
  * equatorial overlaps (Lemma (Inner Product), Lemma (Exponential Sum)):
        b_alpha omega_alpha conj(<phi'_alpha|phi_A>)
          = b_alpha zeta^k 2^{-h/2} 2^{-(n + |v|)/2} i^{-sKs} (-1)^{s.v} (re - i im)
    with re, im the integer parts of Z(B),
where zeta = e^{i pi/4}.  The coefficients of the decompositions in use factor the
same way: every choice of a slot is c_j = r_j g_p zeta^{m_j} with g_p a phase common
to the slot (T: e^{i pi/8}; RZ and CCZ: 1) and an integer m_j, so
  sparsify mode (Lemma (Sparsification)): b_alpha = (||c||_1 / k) G zeta^{M_alpha},
  exact mode:                             b_alpha = (prod_p r_{j_p}) G zeta^{M_alpha},
with G = prod_p g_p.  Terms whose magnitude products prod_p r_{j_p} agree are summed
together with integer arithmetic: sum_alpha zeta^{K_alpha} 2^{-e_alpha/2} is an element
of Z[zeta] / 2^S, held as four Python integers (coordinates of 1, zeta, zeta^2,
zeta^3; zeta^4 = -1; an odd e uses 2^{-1/2} = 2^{-1} (zeta + zeta^7)).  Nothing is
rounded until the one conversion at the end, done in 60-digit decimal arithmetic.

The common factors (||c||_1 / k, the r_j, G) enter as the FP64 values the lowering
produces, so the result is exact up to a relative 1e-16 error in those factors, which
no cancellation between terms can amplify.  This is the exact pin against which the
FP64 oracle and the GPU's FP32 sums state their error per result.
"""
from __future__ import annotations

import cmath
import math
from decimal import Decimal, localcontext

from .chform import popcount
from .decomp import l1_norm, lower
from .estimators import inner_equatorial_parts

_PREC = 60


# ------------------------------ coefficients ------------------------------------
def slot_factors(dec):
    """[(r_j, m_j)] and g for one slot's choices c_j = r_j g zeta^{m_j}, or None when a
    choice's phase relative to the slot's first nonzero choice is not a multiple of
    pi/4."""
    nz = [c for c, _ in dec if c != 0]
    if not nz:
        return None
    g = nz[0] / abs(nz[0])
    out = []
    for c, _ in dec:
        if c == 0:
            out.append((0.0, 0))
            continue
        ang = cmath.phase(c / (abs(c) * g)) / (math.pi / 4)
        m = round(ang)
        if abs(ang - m) > 1e-9:
            return None
        out.append((abs(c), m % 8))
    return out, g


def decomposition_factors(slots):
    """Per slot (choices [(r_j, m_j)], g_p); None if any slot does not factor."""
    out = []
    for dec in slots:
        f = slot_factors(dec)
        if f is None:
            return None
        out.append(f)
    return out


def _mag_key(r: float) -> str:
    return f"{r:.12e}"


def coefficient_parts(factors, choices, mode: str, chi: int, l1: float):
    """(magnitude key, magnitude, M mod 8) of b_alpha / G for the given slot choices."""
    M = 0
    for (ch, _g), j in zip(factors, choices):
        M += ch[j][1]
    if mode == "sparsify":
        return "sparse", l1 / chi, M % 8
    # exact mode: group by the multiset of magnitudes (values equal to 12 digits are
    # the same number written twice, e.g. |c_0| = |c_1| = sqrt2 sin(pi/8) for T)
    counts = {}
    mag = 1.0
    for (ch, _g), j in zip(factors, choices):
        r = ch[j][0]
        k = _mag_key(r)
        counts[k] = counts.get(k, 0) + 1
        mag *= r
    return tuple(sorted(counts.items())), mag, M % 8


def common_phase(factors) -> complex:
    G = 1.0 + 0j
    for _ch, g in factors:
        G *= g
    return G


# ------------------------------ Z[zeta8] accumulator -----------------------------
class Z8Sum:
    """Exact sum of terms s * zeta^K * 2^{-e/2} (s an integer) as four integer
    coordinates over 1, zeta, zeta^2, zeta^3 at the fixed scale 2^-S."""

    def __init__(self, S: int = 512):
        self.S = S
        self.c = [0, 0, 0, 0]

    def _put(self, K: int, val: int):
        K %= 8
        if K >= 4:
            val, K = -val, K - 4
        self.c[K] += val

    def add(self, K: int, e: int, s: int = 1):
        if s == 0:
            return
        if e % 2 == 0:
            sh = self.S - e // 2
            assert sh >= 0, "raise S"
            self._put(K, s << sh)
        else:
            # 2^{-e/2} = 2^{-(e+1)/2} (zeta + zeta^{-1})
            sh = self.S - (e + 1) // 2
            assert sh >= 0, "raise S"
            self._put(K + 1, s << sh)
            self._put(K - 1, s << sh)

    def is_zero(self) -> bool:
        return self.c == [0, 0, 0, 0]

    def decimal(self):
        """(Re, Im) as 60-digit Decimals."""
        with localcontext() as ctx:
            ctx.prec = _PREC
            r2 = Decimal(2).sqrt()
            sc = Decimal(2) ** (-self.S)
            c0, c1, c2, c3 = (Decimal(v) for v in self.c)
            re = (c0 + (c1 - c3) / r2) * sc
            im = (c2 + (c1 + c3) / r2) * sc
            return re, im


def _dmul(a, b):
    """Product of two (Re, Im) Decimal pairs."""
    with localcontext() as ctx:
        ctx.prec = _PREC
        return a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0]


def _dcomplex(z: complex):
    return Decimal(z.real), Decimal(z.imag)


class ExactDecomposition:
    """Coefficient factors of a lowered decomposition, for exact chi-sums."""

    def __init__(self, n: int, ops, chi: int, mode: str, ccz_mode: str = "proj"):
        _, slots = lower(ops, ccz_mode)
        self.factors = decomposition_factors(slots)
        if self.factors is None:
            raise ValueError("a slot's coefficients do not factor as r g zeta^m")
        self.n, self.chi, self.mode = n, chi, mode
        self.l1 = l1_norm(slots)
        self.G = common_phase(self.factors)

    def parts(self, choices):
        return coefficient_parts(self.factors, choices, self.mode, self.chi, self.l1)

    def _finish(self, groups):
        """sum over groups of magnitude * G * (exact Z[zeta8] sum), in Decimal."""
        with localcontext() as ctx:
            ctx.prec = _PREC
            tot = (Decimal(0), Decimal(0))
            for mag, acc in groups.values():
                v = _dmul(acc.decimal(), _dcomplex(self.G))
                m = Decimal(mag)
                tot = (tot[0] + m * v[0], tot[1] + m * v[1])
            return tot

    def amplitude(self, terms, choices, x: int):
        """Exact <x|psi> for the given terms (CHForm) and their slot choices, as
        (Re, Im) Decimals (Eq. (amplitude1) per term)."""
        return self.finish_parts([self.amplitude_parts(terms, choices, x)])

    def amplitude_parts(self, terms, choices, x: int):
        """The exact sum at x over the given terms as {magnitude key: (magnitude,
        integer coordinates)}; parts of disjoint groups of terms add exactly
        (finish_parts)."""
        groups = {}
        for t, ch in zip(terms, choices):
            if t.zero:
                continue
            mu, uu, ww = t.pauli_of(x)
            nv = ~t.v & t.mask
            if (uu ^ t.s) & nv:
                continue
            sign = popcount(uu & ww) + popcount(uu & t.s & t.v)
            key, mag, M = self.parts(ch)
            if key not in groups:
                groups[key] = (mag, Z8Sum())
            groups[key][1].add(M + t.k + 2 * mu + 4 * sign, popcount(t.v) + t.h)
        return {k: (mag, tuple(acc.c)) for k, (mag, acc) in groups.items()}

    def finish_parts(self, parts_list):
        """Merge parts (integer coordinates add exactly), then convert once."""
        merged = {}
        for parts in parts_list:
            for key, (mag, c) in parts.items():
                if key not in merged:
                    merged[key] = (mag, Z8Sum())
                acc = merged[key][1]
                for i in range(4):
                    acc.c[i] += c[i]
        return self._finish(merged)

    def overlap_A(self, terms, choices, A):
        """Exact <phi_A|psi> = sum_alpha b_alpha omega_alpha conj(<phi'_alpha|phi_A>)
        (Lemmas (Norm Estimation), (Inner Product)) as (Re, Im) Decimals."""
        groups = {}
        n = self.n
        for t, ch in zip(terms, choices):
            if t.zero:
                continue
            sKs, sv, nvars, re, im = inner_equatorial_parts(t, A)
            key, mag, M = self.parts(ch)
            if key not in groups:
                groups[key] = (mag, Z8Sum())
            acc = groups[key][1]
            # zeta^{M + k} 2^{-(h + n + |v|)/2} i^{-sKs} (-1)^{sv} (re - i im)
            K = M + t.k - 2 * sKs + 4 * sv
            e = t.h + n + nvars
            acc.add(K, e, re)
            acc.add(K + 6, e, im)       # -i im = zeta^6 im
        return self._finish(groups)

    def eta(self, terms, choices, A):
        """Exact 2^n |<phi_A|psi>|^2 as a Decimal."""
        re, im = self.overlap_A(terms, choices, A)
        with localcontext() as ctx:
            ctx.prec = _PREC
            return (Decimal(2) ** self.n) * (re * re + im * im)


def to_complex(z) -> complex:
    return complex(float(z[0]), float(z[1]))


def abs_decimal(z):
    with localcontext() as ctx:
        ctx.prec = _PREC
        return (z[0] * z[0] + z[1] * z[1]).sqrt()

