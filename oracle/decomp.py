"""Sum-over-Cliffords decompositions and sparsification (oracle; test only).

Sec. 2.3.2 ("Sum-over-Cliffords method") of arXiv:1808.00128 writes each
non-Clifford gate as V = sum_j c_j K_j with Clifford (or, for the exact CCZ
form below, projective) K_j and expands the circuit
U = D_m V_m ... V_1 D_0 into sum over choices (j_1..j_m) of
(prod_p c_{j_p}) D_m K_{j_m} ... K_{j_1} D_0.  Lemma (Sparsification) in
Sec. 5.2 replaces the full sum by k i.i.d. draws j_p ~ |c_j| / ||c||_1 with
equal weights ||c||_1 / k times the phases c_j / |c_j|.

Readings taken here:
  * T = diag(1, e^{i pi/4}) = e^{i pi/8} R(pi/4), R(theta) = exp(-i theta Z / 2);
    the global phase is kept so amplitudes match the dense vector.
  * R(theta) = (cos(theta/2) - sin(theta/2)) I + sqrt2 e^{-i pi/4} sin(theta/2) S
    (Eq. (Rtheta)); for theta < 0 the complex conjugate on (I, S^dagger) is used.
  * The CCZ prefactor printed as 2/9 in Eq. (CCZ_decomposition) is taken as
    1/6: at |000> the bracket sums to 6, and (8/6)^2 = 16/9 = xi(CCZ).
  * "Exact low-rank" CCZ: CCZ = I - 2 P1_a P1_b P1_c with P1 = (I - Z)/2.
  * Exact mode enumerates the nonzero choices in mixed radix, slot 0 the
    least significant digit; sparsify mode draws slot p of term alpha with
    the uniform rng.uniform(seed, alpha, p) by inverse CDF over the choices in
    index order (first j with u < cumulative weight).
"""
from __future__ import annotations

import cmath
import math

from . import rng
from .chform import CHForm, run_gates


def gate_decomposition(op):
    """[(c_j, K_j gate list)] for one non-Clifford gate tuple."""
    name = op[0]
    if name in ("T", "RZ"):
        q = op[1]
        theta = math.pi / 4 if name == "T" else float(op[2])
        glob = cmath.exp(1j * math.pi / 8) if name == "T" else 1.0
        th = abs(theta)
        c0 = math.cos(th / 2) - math.sin(th / 2)
        c1 = math.sqrt(2) * cmath.exp(-1j * math.pi / 4) * math.sin(th / 2)
        if theta >= 0:
            return [(glob * c0, []), (glob * c1, [("S", q)])]
        return [(glob * c0, []), (glob * c1.conjugate(), [("SDG", q)])]
    if name == "CCZ_SUM8":
        a, b, c = op[1], op[2], op[3]
        w = 1.0 / 6.0
        return [
            (w, []),
            (w, [("CZ", a, b)]),
            (w, [("CZ", a, c)]),
            (w, [("CZ", b, c)]),
            (w, [("CZ", a, b), ("CZ", a, c), ("Z", a)]),
            (w, [("CZ", a, b), ("CZ", b, c), ("Z", b)]),
            (w, [("CZ", a, c), ("CZ", b, c), ("Z", c)]),
            (-w, [("CZ", a, b), ("CZ", a, c), ("CZ", b, c), ("Z", a), ("Z", b), ("Z", c)]),
        ]
    if name == "CCZ_PROJ":
        a, b, c = op[1], op[2], op[3]
        return [(1.0, []), (-2.0, [("P1", a), ("P1", b), ("P1", c)])]
    raise ValueError(f"not a non-Clifford gate: {op}")


def lower(ops, ccz_mode: str = "proj"):
    """Split a circuit into Clifford gates and slots.

    Returns (gates, slots): gates holds Clifford tuples and ('SLOT', p);
    slots[p] is the decomposition list of slot p.
    """
    gates, slots = [], []
    for op in ops:
        if op[0] in ("T", "RZ"):
            gates.append(("SLOT", len(slots)))
            slots.append(gate_decomposition(op))
        elif op[0] == "CCZ":
            kind = "CCZ_PROJ" if ccz_mode == "proj" else "CCZ_SUM8"
            gates.append(("SLOT", len(slots)))
            slots.append(gate_decomposition((kind,) + tuple(op[1:])))
        else:
            gates.append(op)
    return gates, slots


def lower_gadget(n: int, ops, ccz_mode: str = "proj"):
    """Fixed-sample gadget form (Sec. 2.3.1, Eqs. (singlegate), (Uidentity)).

    Every non-Clifford gate V_j on t_j qubits gets t_j ancilla qubits (numbered from
    n on, in the order of the gates) holding the magic state |V_j> = V_j |+^t_j>; the
    gate itself becomes CNOT(q_k -> a_k) for its qubits q_k and ancillas a_k, and
    every ancilla is post-selected on 0 by the projector (I + Z)/2.  Then
    U|0^n> = 2^{tau/2} (1 x <0^tau|) C |0^n>|Psi>; the factor 2^{t_j/2} of each gadget
    is folded into the coefficients of its magic-state slot, so that the final
    (n + tau)-qubit state is exactly U|0^n> (x) |0^tau>.  The magic states take the
    sum-over-Cliffords decompositions of V_j applied to |+^t_j>.

    Returns (n_total, gates, slots) in the form of lower().
    """
    gadgets, a = [], n
    for op in ops:
        if op[0] in ("T", "RZ"):
            gadgets.append((op, [a]))
            a += 1
        elif op[0] == "CCZ":
            gadgets.append((op, [a, a + 1, a + 2]))
            a += 3
    gates, slots = [], []
    for op, anc in gadgets:
        for q in anc:
            gates.append(("H", q))
        if op[0] == "CCZ":
            vop = ("CCZ_PROJ" if ccz_mode == "proj" else "CCZ_SUM8",) + tuple(anc)
        else:
            vop = (op[0], anc[0]) + tuple(op[2:])
        scale = 2.0 ** (len(anc) / 2)
        gates.append(("SLOT", len(slots)))
        slots.append([(c * scale, K) for c, K in gate_decomposition(vop)])
    k = 0
    for op in ops:
        if op[0] in ("T", "RZ", "CCZ"):
            anc = gadgets[k][1]
            k += 1
            for qk, ak in zip(op[1:1 + len(anc)], anc):
                gates.append(("CX", qk, ak))
        else:
            gates.append(op)
    for q in range(n, a):
        gates.append(("P0", q))
    return a, gates, slots


def l1_norm(slots) -> float:
    """||c||_1 of the product decomposition = prod_p ||c^(p)||_1 (Sec. 2.3.2)."""
    out = 1.0
    for dec in slots:
        out *= sum(abs(c) for c, _ in dec)
    return out


def exact_chi(slots) -> int:
    out = 1
    for dec in slots:
        out *= sum(1 for c, _ in dec if c != 0)
    return out


def choices_exact(slots, alpha: int):
    """Mixed-radix digits of term alpha over the nonzero choices of each slot."""
    out = []
    for dec in slots:
        nz = [j for j, (c, _) in enumerate(dec) if c != 0]
        out.append(nz[alpha % len(nz)])
        alpha //= len(nz)
    return out


def choice_sparsify(dec, u: float) -> int:
    """Inverse CDF of p_j = |c_j| / ||c||_1 (proof of Lemma (Sparsification))."""
    norm = sum(abs(c) for c, _ in dec)
    acc = 0.0
    last = None
    for j, (c, _) in enumerate(dec):
        if c == 0:
            continue
        last = j
        acc += abs(c) / norm
        if u < acc:
            return j
    return last


def choices_sparsify(slots, alpha: int, seed: int):
    return [choice_sparsify(dec, rng.uniform(seed, alpha, p)) for p, dec in enumerate(slots)]


def coefficient(slots, choices, mode: str, chi: int) -> complex:
    """b_alpha: prod c_{j_p} (exact) or (||c||_1/k) prod c_{j_p}/|c_{j_p}| (sparsify)."""
    if mode == "exact":
        b = 1.0 + 0j
        for dec, j in zip(slots, choices):
            b *= dec[j][0]
        return b
    b = l1_norm(slots) / chi + 0j
    for dec, j in zip(slots, choices):
        c = dec[j][0]
        b *= c / abs(c)
    return b


def term_gates(gates, slots, choices):
    """The Clifford/projector gate list of one term."""
    out = []
    for g in gates:
        if g[0] == "SLOT":
            out.extend(slots[g[1]][choices[g[1]]][1])
        else:
            out.append(g)
    return out


def build_term(n: int, gates, slots, choices) -> CHForm:
    return run_gates(n, term_gates(gates, slots, choices))


def term_choices(slots, alpha: int, mode: str, seed: int):
    if mode == "exact":
        return choices_exact(slots, alpha)
    return choices_sparsify(slots, alpha, seed)


def build_decomposition(n: int, ops, chi: int, mode: str, seed: int = 0, ccz_mode: str = "proj",
                        alphas=None, method: str = "sum"):
    """Terms (CHForm) and coefficients b_alpha of the stabilizer decomposition.

    `alphas` restricts the work to a subset of term indices (the other terms
    are not built); chi is still the total number of terms.  method "gadget" builds
    the fixed-sample gadget form on n + tau qubits (lower_gadget).
    """
    if method == "gadget":
        n, gates, slots = lower_gadget(n, ops, ccz_mode)
    else:
        gates, slots = lower(ops, ccz_mode)
    if mode == "exact" and chi != exact_chi(slots):
        raise ValueError(f"exact mode needs chi = {exact_chi(slots)}")
    alphas = range(chi) if alphas is None else alphas
    terms, coefs, chs = [], [], []
    for a in alphas:
        ch_ = term_choices(slots, a, mode, seed)
        chs.append(ch_)
        terms.append(build_term(n, gates, slots, ch_))
        coefs.append(coefficient(slots, ch_, mode, chi))
    return terms, coefs, chs
