"""The identity behind the norm kernel's change-of-variables route, checked by brute
force on small random CH-form data (no GPU, independent of both the kernel and the
oracle): for invertible F with G = F^{-T} (so F G^T = I), symmetric D with Z4
diagonal, any v and s,

    sum_{x in Z2^n, x = 0 off v} i^{x^T K x + 2 (s.x + s^T K x)},   K = G^T D G,

equals the sum over y in Z2^n with (F^T y)_k = 0 for k not in v of
i^{y^T D y + 2 (F s + D G s).y}, and substituting the reduced constraints
y_p = h.y one by one (diagonal carries, rank-2 row updates) leaves a form on the
remaining variables with the same sum."""
import random

import pytest


def _par(x):
    return bin(x).count("1") & 1


def _bit(x, j):
    return (x >> j) & 1


def _matvec(rows, x):
    return sum(_par(r & x) << c for c, r in enumerate(rows))


def _rank_full(rows, n):
    r, rank = list(rows), 0
    for col in range(n):
        piv = next((i for i in range(rank, n) if _bit(r[i], col)), None)
        if piv is None:
            continue
        r[rank], r[piv] = r[piv], r[rank]
        for i in range(n):
            if i != rank and _bit(r[i], col):
                r[i] ^= r[rank]
        rank += 1
    return rank == n


def _inverse(rows, n):
    r = [rows[i] | (1 << (n + i)) for i in range(n)]
    for col in range(n):
        piv = next(i for i in range(col, n) if _bit(r[i], col))
        r[col], r[piv] = r[piv], r[col]
        for i in range(n):
            if i != col and _bit(r[i], col):
                r[i] ^= r[col]
    return [x >> n for x in r]


def _transpose(rows, n):
    return [sum(_bit(rows[c], k) << c for c in range(n)) for k in range(n)]


def _sum_x(n, Doff, dd, G, v, s):
    z0 = _matvec(G, s)
    Dfull = [Doff[c] | ((dd[c] & 1) << c) for c in range(n)]
    tot = 0
    for xs in range(1 << n):
        if xs & ~v:
            continue
        y = _matvec(G, xs)
        q = sum(dd[c] for c in range(n) if _bit(y, c))
        q += 2 * sum(_bit(Doff[c], d) for c in range(n) for d in range(c + 1, n) if _bit(y, c) and _bit(y, d))
        q += 2 * (_par(s & xs) ^ _par(z0 & _matvec(Dfull, y)))
        tot += 1j ** (q % 4)
    return tot


def _sum_folded(n, Doff, dd, F, G, v, s):
    nmask = (1 << n) - 1
    z0, u = _matvec(G, s), _matvec(F, s)
    Dfull = [Doff[c] | ((dd[c] & 1) << c) for c in range(n)]
    odd = sum((dd[c] & 1) << c for c in range(n))
    Lb = sum(((dd[c] >> 1) & 1) << c for c in range(n)) ^ u ^ _matvec(Dfull, z0)
    act, Q = nmask, list(Doff)
    fs = [f for k, f in enumerate(_transpose(F, n)) if not _bit(v, k)]
    piv = []
    for i in range(len(fs)):
        p = (fs[i] & -fs[i]).bit_length() - 1
        piv.append(p)
        for j in range(len(fs)):
            if j != i and _bit(fs[j], p):
                fs[j] ^= fs[i]
    for p, f in zip(piv, fs):
        h = f & ~(1 << p)
        q = Q[p] & act & ~(1 << p)
        op, lp = _bit(odd, p), _bit(Lb, p)
        Lb ^= h & ((-lp & nmask) ^ (odd if op else 0) ^ q)
        if op:
            odd ^= h
        for c in range(n):
            if _bit(h | q, c):
                Q[c] ^= (q if _bit(h, c) else 0) ^ (h if _bit(q, c) else 0) ^ \
                        ((h & ~(1 << c)) if (op and _bit(h, c)) else 0)
        act &= ~(1 << p)
    vars_ = [c for c in range(n) if _bit(act, c)]
    tot = 0
    for bits in range(1 << len(vars_)):
        y = sum(((bits >> i) & 1) << c for i, c in enumerate(vars_))
        q = bin(odd & y).count("1") + 2 * bin(Lb & y).count("1")
        q += 2 * sum(_bit(Q[c], d) for c in vars_ for d in vars_ if c < d and _bit(y, c) and _bit(y, d))
        tot += 1j ** (q % 4)
    return tot


@pytest.mark.parametrize("seed", range(6))
def test_change_of_variables_matches_direct_sum(seed):
    rng = random.Random(1000 + seed)
    for _ in range(40):
        n = rng.randint(1, 6)
        while True:
            F = [rng.getrandbits(n) for _ in range(n)]
            if _rank_full(F, n):
                break
        G = _transpose(_inverse(F, n), n)
        assert all(_par(F[i] & G[j]) == (i == j) for i in range(n) for j in range(n))   # F G^T = I
        Doff = [0] * n
        for c in range(n):
            for d in range(c + 1, n):
                if rng.getrandbits(1):
                    Doff[c] |= 1 << d
                    Doff[d] |= 1 << c
        dd = [rng.randrange(4) for _ in range(n)]
        v, s = rng.getrandbits(n), rng.getrandbits(n)
        assert abs(_sum_x(n, Doff, dd, G, v, s) - _sum_folded(n, Doff, dd, F, G, v, s)) < 1e-9
