"""Seeded synthetic workloads: circuits and input batches.

This module only draws circuits and inputs from a seeded numpy generator.  It
holds none of the simulation arithmetic (no decompositions, no tableau rules,
no amplitudes), so both the CUDA path and the CPU oracle may consume it.

A circuit is a list of plain tuples acting on qubits 0..n-1:

    ('H', q)  ('S', q)  ('SDG', q)  ('Z', q)          single-qubit Cliffords
    ('CX', c, t)  ('CZ', a, b)                         two-qubit Cliffords
    ('T', q)                                           diag(1, e^{i pi/4})
    ('RZ', q, theta)                                   exp(-i theta Z / 2)
    ('CCZ', a, b, c)                                   doubly controlled Z

Basis strings are n-bit integers with bit j holding qubit j.

The workload shapes follow the paper's experiments: random Clifford+T
circuits, QAOA on Max-E3LIN2 (Sec. 2.4.1) and the hidden-shift circuits
(Sec. 2.4.2), whose exact instances are not published in the paper; these
generators are seeded stand-ins with the same structure.
"""
from __future__ import annotations

import numpy as np

CLIFFORD_1Q = ("H", "S", "SDG", "Z")
CLIFFORD_2Q = ("CX", "CZ")
NON_CLIFFORD = ("T", "RZ", "CCZ")


def random_clifford_t(n: int, n_clifford: int, n_t: int, seed: int):
    """Random Clifford+T circuit.

    Each Clifford gate is uniform over {H, S, CX, CZ}; single-qubit gates pick a
    uniform qubit, two-qubit gates a uniform ordered pair of distinct qubits.
    The n_t T gates sit at uniform distinct positions among the
    n_clifford + n_t gate slots, each on a uniform qubit.
    """
    rng = np.random.default_rng(seed)
    total = n_clifford + n_t
    t_pos = set(int(p) for p in rng.choice(total, size=n_t, replace=False)) if n_t else set()
    ops = []
    for pos in range(total):
        if pos in t_pos:
            ops.append(("T", int(rng.integers(n))))
            continue
        kind = int(rng.integers(4))
        if kind == 0:
            ops.append(("H", int(rng.integers(n))))
        elif kind == 1:
            ops.append(("S", int(rng.integers(n))))
        else:
            if n < 2:
                ops.append(("H", 0))
                continue
            a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
            ops.append(("CX" if kind == 2 else "CZ", a, b))
    return ops


def e3lin2_instance(n: int, degree: int, seed: int, max_tries: int = 10000):
    """Random Max-E3LIN2 instance by a configuration model.

    Every variable is listed `degree` times, the list is shuffled and cut into
    triples; a shuffle is rejected if a triple repeats a variable or two triples
    coincide.  Leftover stubs (n*degree mod 3) are dropped, so up to two
    variables end with a lower degree.  Signs d are uniform +-1.
    Returns a list of ((u, v, w), d) with u < v < w.
    """
    rng = np.random.default_rng(seed)
    stubs = np.repeat(np.arange(n), degree)
    m = len(stubs) // 3
    for _ in range(max_tries):
        perm = rng.permutation(stubs)[: 3 * m].reshape(m, 3)
        triples = [tuple(sorted(int(x) for x in row)) for row in perm]
        if any(len(set(t)) < 3 for t in triples):
            continue
        if len(set(triples)) < m:
            continue
        signs = rng.choice(np.array([-1, 1]), size=m)
        return [(t, int(d)) for t, d in zip(triples, signs)]
    raise RuntimeError("configuration model did not converge")


def qaoa_e3lin2_circuit(n: int, degree: int, gamma: float, beta: float, seed: int):
    """QAOA p=1 circuit exp(-i beta B) exp(-i gamma C) H^n for Max-E3LIN2.

    C = 1/2 sum d_uvw Z_u Z_v Z_w; each term is
    CX(u,w) CX(v,w) RZ_w(gamma*d) CX(v,w) CX(u,w).  The mixer on every qubit is
    exp(-i beta X) = H RZ(2 beta) H.
    Returns (ops, instance).
    """
    inst = e3lin2_instance(n, degree, seed)
    ops = [("H", q) for q in range(n)]
    for (u, v, w), d in inst:
        ops += [("CX", u, w), ("CX", v, w), ("RZ", w, gamma * d), ("CX", v, w), ("CX", u, w)]
    for q in range(n):
        ops += [("H", q), ("RZ", q, 2.0 * beta), ("H", q)]
    return ops, inst


def hidden_shift_circuit(n: int, n_ccz: int, seed: int):
    """Hidden-shift circuit for a Maiorana-McFarland bent function.

    Qubits 0..h-1 hold x, h..2h-1 hold y (n = 2h).  f(x, y) = x.y + g(y) with
    g the XOR of n_ccz/2 seeded cubic monomials; its dual is
    f~(x, y) = x.y + g(x).  The circuit
        H^n, O_f, H^n, Z(s), O_f~, H^n
    maps |0^n> to |s> for a uniform random shift s.  Each phase oracle is h CZ
    gates plus n_ccz/2 CCZ gates.  Returns (ops, s).
    """
    if n % 2 or n_ccz % 2:
        raise ValueError("n and n_ccz must be even")
    h = n // 2
    rng = np.random.default_rng(seed)
    monos = []
    seen = set()
    while len(monos) < n_ccz // 2:
        t = tuple(sorted(int(x) for x in rng.choice(h, size=3, replace=False)))
        if t not in seen:
            seen.add(t)
            monos.append(t)
    s = int(rng.integers(0, np.iinfo(np.uint64).max, dtype=np.uint64, endpoint=True))
    s &= (1 << n) - 1
    ops = [("H", q) for q in range(n)]
    ops += [("CZ", i, h + i) for i in range(h)]
    ops += [("CCZ", h + a, h + b, h + c) for a, b, c in monos]
    ops += [("H", q) for q in range(n)]
    ops += [("Z", q) for q in range(n) if (s >> q) & 1]
    ops += [("CZ", i, h + i) for i in range(h)]
    ops += [("CCZ", a, b, c) for a, b, c in monos]
    ops += [("H", q) for q in range(n)]
    return ops, s


def random_bitstrings(n: int, count: int, seed: int) -> np.ndarray:
    """`count` uniform n-bit strings as uint64."""
    rng = np.random.default_rng(seed)
    words = rng.integers(0, np.iinfo(np.uint64).max, size=count, dtype=np.uint64, endpoint=True)
    if n < 64:
        words &= np.uint64((1 << n) - 1)
    return words


def count_ops(ops):
    """Histogram of gate names."""
    hist = {}
    for op in ops:
        hist[op[0]] = hist.get(op[0], 0) + 1
    return hist


# Named configurations (sizes of the paper's workloads; see the module doc).
SEED_BASE = 180800128


def config_tiny():
    """n=10, 200 random Cliffords + 6 T; exact 2-term T -> chi = 64."""
    ops = random_clifford_t(10, 200, 6, SEED_BASE + 1)
    return dict(name="clifford_t_n10_t6_exact", n=10, ops=ops, chi=64, mode="exact", seed=0,
                batch=1024, L=64)


def config_mid():
    """n=40, 2000 random Cliffords + 24 T; sparsified to chi = 2^16."""
    ops = random_clifford_t(40, 2000, 24, SEED_BASE + 2)
    return dict(name="clifford_t_n40_t24_chi65536", n=40, ops=ops, chi=1 << 16,
                mode="sparsify", seed=SEED_BASE + 12, batch=4096, L=256, chains=256)


def config_hidden_shift():
    """n=40 hidden shift with 16 CCZ; exact projector form of CCZ -> chi = 2^16."""
    ops, s = hidden_shift_circuit(40, 16, SEED_BASE + 3)
    return dict(name="hidden_shift_n40_ccz16", n=40, ops=ops, chi=1 << 16, mode="exact", seed=0,
                shift=s, chains=1024, batch=4096, L=256)


def config_qaoa(beta: float = 0.2, chi: int = 1 << 20):
    """n=50 QAOA p=1 on Max-E3LIN2 (degree 4), gamma=0.3."""
    ops, inst = qaoa_e3lin2_circuit(50, 4, 0.3, beta, SEED_BASE + 4)
    return dict(name="qaoa_e3lin2_n50", n=50, ops=ops, chi=chi, mode="sparsify",
                seed=SEED_BASE + 14, instance=inst, chains=256, steps=10000, L=512)
