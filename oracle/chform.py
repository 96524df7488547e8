"""CH-form stabilizer states (oracle; test infrastructure only).

Follows Sec. 4.1 ("Phase-sensitive Clifford simulator") of arXiv:1808.00128.
Equations are cited by their LaTeX labels, e.g. Eq. (H2).

A state is |phi> = omega U_C U_H |s>  (Eq. (phi)) with
  U_C^{-1} Z_p U_C = prod_j Z_j^{G[p,j]}
  U_C^{-1} X_p U_C = i^{gamma_p} prod_j X_j^{F[p,j]} Z_j^{M[p,j]}   (Eq. (tableaux))
  U_H = H(v)                                                         (Eq. (Htype))
Rows are Python ints: bit j of F[p] is F[p, j].  omega is kept exactly as
(zero, k, h) meaning 0 if zero else exp(i pi k / 4) * 2^(-h/2).

Readings of the paper taken here (the GPU path takes the same ones):
  * the update rules of one gate are simultaneous (right-hand sides use the
    values before the gate);
  * the incoming omega is multiplied into the new omega of Eqs. (H1), (H7);
  * "the first qubit" of V_b in the proof of Prop. (prop:H) is the lowest index;
  * the single-qubit rewrite omega1 S^a H^b |c> picks a = 0 whenever b = 0
    (the two choices describe the same state);
  * a projective gate (I + (-1)^sigma Z_j)/2 whose result vanishes marks the
    term as zero.
"""
from __future__ import annotations

import cmath
import math


def bit(x: int, j: int) -> int:
    return (x >> j) & 1


def popcount(x: int) -> int:
    return bin(x).count("1")


def bits_of(x: int):
    j = 0
    while x:
        if x & 1:
            yield j
        x >>= 1
        j += 1


class CHForm:
    """Phase-sensitive CH-form of one n-qubit stabilizer state (n <= 64)."""

    def __init__(self, n: int):
        # Initial state |0^n>: G = F = I, M = 0, gamma = v = s = 0 (Sec. 4.1,
        # "Simulation of unitary gates").
        self.n = n
        self.mask = (1 << n) - 1
        self.F = [1 << p for p in range(n)]
        self.G = [1 << p for p in range(n)]
        self.M = [0] * n
        self.gamma = [0] * n
        self.v = 0
        self.s = 0
        self.zero = False
        self.k = 0
        self.h = 0

    def copy(self) -> "CHForm":
        c = CHForm.__new__(CHForm)
        c.n, c.mask = self.n, self.mask
        c.F, c.G, c.M, c.gamma = list(self.F), list(self.G), list(self.M), list(self.gamma)
        c.v, c.s, c.zero, c.k, c.h = self.v, self.s, self.zero, self.k, self.h
        return c

    def omega(self) -> complex:
        if self.zero:
            return 0j
        return cmath.exp(1j * math.pi * (self.k % 8) / 4) * 2.0 ** (-self.h / 2)

    # ---------------- left multiplication U_C <- Gamma U_C (Sec. 4.1 rules) ---------
    def left_S(self, q: int):
        """L[S_q]: M[q,p] ^= G[q,p] for all p; gamma_q -= 1."""
        for p in range(self.n):
            self.M[q] ^= bit(self.G[q], p) << p
        self.gamma[q] = (self.gamma[q] - 1) % 4

    def left_CZ(self, q: int, r: int):
        """L[CZ_{q,r}]: M[q,p] ^= G[r,p]; M[r,p] ^= G[q,p]."""
        Gq, Gr = self.G[q], self.G[r]
        for p in range(self.n):
            self.M[q] ^= bit(Gr, p) << p
            self.M[r] ^= bit(Gq, p) << p

    def left_CX(self, q: int, r: int):
        """L[CX_{q,r}]: G[r,p] ^= G[q,p]; F[q,p] ^= F[r,p]; M[q,p] ^= M[r,p];
        gamma_q += gamma_r + 2 (M F^T)_{q,r}, with the pre-gate M."""
        MFt_qr = sum(bit(self.M[q], j) * bit(self.F[r], j) for j in range(self.n))
        new_gamma_q = (self.gamma[q] + self.gamma[r] + 2 * MFt_qr) % 4
        Gq, Fr, Mr = self.G[q], self.F[r], self.M[r]
        for p in range(self.n):
            self.G[r] ^= bit(Gq, p) << p
            self.F[q] ^= bit(Fr, p) << p
            self.M[q] ^= bit(Mr, p) << p
        self.gamma[q] = new_gamma_q

    # ---------------- right multiplication U_C <- U_C Gamma (Sec. 4.1 rules) --------
    def right_S(self, q: int):
        """R[S_q]: M[p,q] ^= F[p,q]; gamma_p -= F[p,q]."""
        for p in range(self.n):
            f = bit(self.F[p], q)
            self.M[p] ^= f << q
            self.gamma[p] = (self.gamma[p] - f) % 4

    def right_CZ(self, q: int, r: int):
        """R[CZ_{q,r}]: M[p,q] ^= F[p,r]; M[p,r] ^= F[p,q]; gamma_p += 2 F[p,q] F[p,r]."""
        for p in range(self.n):
            fq, fr = bit(self.F[p], q), bit(self.F[p], r)
            self.M[p] ^= (fr << q) ^ (fq << r)
            self.gamma[p] = (self.gamma[p] + 2 * fq * fr) % 4

    def right_CX(self, q: int, r: int):
        """R[CX_{q,r}]: G[p,q] ^= G[p,r]; F[p,r] ^= F[p,q]; M[p,q] ^= M[p,r]."""
        for p in range(self.n):
            self.G[p] ^= bit(self.G[p], r) << q
            self.F[p] ^= bit(self.F[p], q) << r
            self.M[p] ^= bit(self.M[p], r) << q

    # ---------------- gates ----------------------------------------------------------
    def apply_S(self, q):
        self.left_S(q)

    def apply_SDG(self, q):
        for _ in range(3):
            self.left_S(q)

    def apply_Z(self, q):
        for _ in range(2):
            self.left_S(q)

    def apply_CZ(self, q, r):
        self.left_CZ(q, r)

    def apply_CX(self, q, r):
        self.left_CX(q, r)

    def apply_H(self, p: int):
        """Hadamard on qubit p: Eqs. (H1)-(H7) and Prop. (prop:H)."""
        if self.zero:
            return
        nv = ~self.v & self.mask
        # Eq. (H2)
        t = self.s ^ (self.G[p] & self.v)
        u = self.s ^ (self.F[p] & nv) ^ (self.M[p] & self.v)
        # Eq. (H4)
        alpha = sum(bit(self.G[p], j) * (1 - bit(self.v, j)) * bit(self.s, j) for j in range(self.n)) % 2
        beta = sum(bit(self.M[p], j) * (1 - bit(self.v, j)) * bit(self.s, j)
                   + bit(self.F[p], j) * bit(self.v, j) * (bit(self.M[p], j) + bit(self.s, j))
                   for j in range(self.n)) % 2
        g = self.gamma[p]
        if t == u:
            # omega' = 2^{-1/2} [(-1)^alpha + i^gamma_p (-1)^beta] omega  (Eq. (H1), t = u)
            f = (-1) ** alpha + (1j ** g) * (-1) ** beta
            mag2 = round(abs(f) ** 2)
            assert mag2 == 2, "H with t=u must keep the norm (gamma_p odd)"
            self.k += _phase_index(f / abs(f))
            self.s = t
            return
        # H_p|phi> = 2^{-1/2} (-1)^alpha omega U_C U_H (|t> + i^delta |u>)  (Eqs. (H1), (H6))
        delta = (g + 2 * (alpha + beta)) % 4
        self.k += 4 * alpha
        k1 = self._prop_H(t, u, delta)     # U_H(|t>+i^d|u>) = sqrt2 e^{i pi k1/4} W_C W_H |s'>
        self.k += k1                        # 2^{-1/2} * sqrt2 = 1: h unchanged (Eq. (H7))

    def apply_proj(self, j: int, sigma: int):
        """Projective gate (I + (-1)^sigma Z_j)/2 (Sec. 4.1, end)."""
        if self.zero:
            return
        # U_C^{-1} Z_j U_C = Z(G_j); Z(G_j) U_H |s> = (-1)^{alpha'} U_H |s ^ (G_j & v)>
        nv = ~self.v & self.mask
        t = self.s ^ (self.G[j] & self.v)
        alpha = popcount(self.G[j] & nv & self.s) % 2
        sign = (sigma + alpha) % 2
        if t == self.s:
            if sign:
                self.zero = True       # (1 - 1)|s> = 0
            return                     # (1/2)(1 + 1)|s> = |s>
        delta = 2 * sign
        k1 = self._prop_H(self.s, t, delta)
        self.k += k1
        self.h += 1                    # (1/2) * sqrt2

    def _prop_H(self, t: int, u: int, delta: int) -> int:
        """Prop. (prop:H): U_H(|t> + i^delta |u>) = omega1 W_C W_H |s'>, t != u.

        Updates U_C <- U_C W_C (right multiplications), v, s.  Returns k1 with
        omega1 = sqrt(2) exp(i pi k1 / 4).
        """
        d = t ^ u
        V0 = d & ~self.v & self.mask
        V1 = d & self.v
        if V0:
            q = min(bits_of(V0))
            for i in bits_of(V0):
                if i != q:
                    self.right_CX(q, i)
            for i in bits_of(V1):
                self.right_CZ(q, i)
        else:
            q = min(bits_of(V1))
            for i in bits_of(V1):
                if i != q:
                    self.right_CX(i, q)
        if bit(t, q):
            y, z = u ^ (1 << q), u
        else:
            y, z = t, t ^ (1 << q)
        a, b, c, k1 = single_qubit_form(bit(self.v, q), bit(y, q), bit(z, q), delta)
        if a:
            self.right_S(q)
        self.v = (self.v & ~(1 << q)) | (b << q)
        self.s = (y & ~(1 << q)) | (c << q)
        return k1

    # ---------------- measurements (Eqs. (amplitude), (amplitude1)) -----------------
    def pauli_of(self, x: int):
        """Q = prod_{p: x_p=1} U_C^{-1} X_p U_C written as i^mu X(u) Z(w)."""
        mu, uu, ww = 0, 0, 0
        for p in range(self.n):
            if bit(x, p):
                # (i^mu X(u) Z(w)) (i^g X(F_p) Z(M_p)) = i^{mu+g} (-1)^{w.F_p} X(u^F_p) Z(w^M_p)
                mu = (mu + self.gamma[p] + 2 * popcount(ww & self.F[p])) % 4
                uu ^= self.F[p]
                ww ^= self.M[p]
        return mu, uu, ww

    def amplitude_from_pauli(self, mu: int, uu: int, ww: int) -> complex:
        """<0^n| i^mu X(u) Z(w) U_H |s> times omega (Eq. (amplitude1))."""
        if self.zero:
            return 0j
        nv = ~self.v & self.mask
        if (uu ^ self.s) & nv:
            return 0j
        sign = popcount(uu & ww) + popcount(uu & self.s & self.v)
        ph = (2 * mu + 4 * sign + self.k) % 8
        return cmath.exp(1j * math.pi * ph / 4) * 2.0 ** (-(popcount(self.v) + self.h) / 2)

    def amplitude(self, x: int) -> complex:
        """<x|phi>."""
        return self.amplitude_from_pauli(*self.pauli_of(x))

    def sample(self, flips: int) -> int:
        """Sample x from |<x|phi>|^2 (Sec. 4.1, "Simulating measurements").

        `flips` supplies the random bits: w = s, bit j of w flipped when v_j = 1
        and bit j of `flips` is set; x = w G^T (mod 2).
        """
        w = self.s ^ (flips & self.v)
        x = 0
        for j in range(self.n):
            x |= (popcount(w & self.G[j]) & 1) << j
        return x

    def key(self):
        """Canonical tuple for bit-exact comparisons."""
        return (tuple(self.F), tuple(self.G), tuple(self.M), tuple(self.gamma), self.v,
                self.s, self.zero, (self.k % 8) if not self.zero else 0,
                self.h if not self.zero else 0)


def _phase_index(z: complex) -> int:
    """k with z = exp(i pi k / 4); asserts z is an 8th root of unity."""
    ang = cmath.phase(z) / (math.pi / 4)
    k = round(ang)
    assert abs(ang - k) < 1e-9, z
    return k % 8


def single_qubit_form(vq: int, yq: int, zq: int, delta: int):
    """Find (a, b, c, k1) with H^{vq}(|yq> + i^delta |zq>) = sqrt2 e^{i pi k1/4} S^a H^b |c>.

    Brute force over the eight (a, b, c), a = 0 tried first (proof of
    Prop. (prop:H)).
    """
    r2 = 1 / math.sqrt(2)
    Hm = ((r2, r2), (r2, -r2))

    def apply(mat, vec):
        return (mat[0][0] * vec[0] + mat[0][1] * vec[1], mat[1][0] * vec[0] + mat[1][1] * vec[1])

    vec = [0j, 0j]
    vec[yq] += 1
    vec[zq] += 1j ** delta
    vec = tuple(vec)
    if vq:
        vec = apply(Hm, vec)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                cand = (1.0 + 0j, 0j) if c == 0 else (0j, 1.0 + 0j)
                if b:
                    cand = apply(Hm, cand)
                if a:
                    cand = (cand[0], 1j * cand[1])
                # vec = w * cand ?
                inner = vec[0] * cand[0].conjugate() + vec[1] * cand[1].conjugate()
                resid = (vec[0] - inner * cand[0], vec[1] - inner * cand[1])
                if abs(resid[0]) < 1e-12 and abs(resid[1]) < 1e-12:
                    assert abs(abs(inner) - math.sqrt(2)) < 1e-12
                    return a, b, c, _phase_index(inner / abs(inner))
    raise AssertionError("no CH single-qubit form found")


def run_gates(n: int, gates, ch: CHForm | None = None) -> CHForm:
    """Apply a list of Clifford/projector gate tuples to |0^n> (or `ch`)."""
    ch = ch if ch is not None else CHForm(n)
    for g in gates:
        name = g[0]
        if name == "H":
            ch.apply_H(g[1])
        elif name == "S":
            ch.apply_S(g[1])
        elif name == "SDG":
            ch.apply_SDG(g[1])
        elif name == "Z":
            ch.apply_Z(g[1])
        elif name == "X":
            ch.apply_H(g[1]); ch.apply_Z(g[1]); ch.apply_H(g[1])
        elif name == "CX":
            ch.apply_CX(g[1], g[2])
        elif name == "CZ":
            ch.apply_CZ(g[1], g[2])
        elif name == "P0":
            ch.apply_proj(g[1], 0)
        elif name == "P1":
            ch.apply_proj(g[1], 1)
        else:
            raise ValueError(f"not a Clifford/projector gate: {g}")
    return ch
