"""Pins for the oracle exponential sum (Lemma (Exponential Sum), Sec. 4.3)."""
import itertools
import random

import pytest

from oracle.expsum import expsum, expsum_z2


def brute(B):
    m = len(B)
    z = 0j
    for x in itertools.product((0, 1), repeat=m):
        q = sum(x[a] * B[a][b] * x[b] for a in range(m) for b in range(m)) % 4
        z += 1j ** q
    return z


def rand_B(m, rng):
    B = [[0] * m for _ in range(m)]
    for a in range(m):
        B[a][a] = rng.randrange(4)
        for b in range(a + 1, m):
            B[a][b] = B[b][a] = rng.randrange(2)
    return B


@pytest.mark.parametrize("m", list(range(0, 11)))
def test_expsum_brute_force(m):
    rng = random.Random(100 + m)
    for _ in range(60 if m < 8 else 15):
        B = rand_B(m, rng)
        re, im = expsum(B)
        z = brute(B)
        assert complex(re, im) == pytest.approx(z, abs=1e-9)


def test_expsum_negative_value():
    """n = 1, B = 3: 1 + i^3 = 1 - i (the lemma's alpha, beta must allow -1)."""
    assert expsum([[3]]) == (1, -1)
    assert expsum([[2]]) == (0, 0)
    assert expsum([[1]]) == (1, 1)
    assert expsum([[0]]) == (2, 0)
    assert expsum([]) == (1, 0)


def test_identity_two_variables():
    """sum_{x1,x2} (-1)^{x1 x2 + mu1 x1 + mu2 x2} = 2 (-1)^{mu1 mu2}  (Eq. (identity))."""
    for mu1 in (0, 1):
        for mu2 in (0, 1):
            got = expsum_z2([[0, 1], [0, 0]], [mu1, mu2])
            assert got == 2 * (-1) ** (mu1 * mu2)


def test_z2_nonsymmetric_brute():
    rng = random.Random(7)
    for _ in range(200):
        n = rng.randrange(0, 8)
        M = [[rng.randrange(2) for _ in range(n)] for _ in range(n)]
        L = [rng.randrange(2) for _ in range(n)]
        want = sum((-1) ** ((sum(x[a] * M[a][b] * x[b] for a in range(n) for b in range(n))
                             + sum(L[a] * x[a] for a in range(n))) % 2)
                   for x in itertools.product((0, 1), repeat=n))
        assert expsum_z2(M, L) == want


def test_magnitude_is_power_of_two():
    rng = random.Random(8)
    for _ in range(300):
        re, im = expsum(rand_B(rng.randrange(0, 9), rng))
        for part in (re, im):
            assert part == 0 or (abs(part) & (abs(part) - 1)) == 0
        if re and im:
            assert abs(re) == abs(im)
