"""Exponential sums Z(B) = sum_x i^{x B x^T} (oracle; test infrastructure only).

Follows Lemma (Exponential Sum) and its proof in Sec. 4.3 of arXiv:1808.00128:
the Z4-valued form is lifted to a Z2-valued form on one more variable
(Eqs. (Q), (real)), and each Z2 sum is reduced two variables at a time
(Eqs. (Zreal), (eq1partialsum), (identity), (eq5)).

Reading taken here: the lemma states alpha, beta in {0, 1}, but Z(B) can be
negative (n = 1, B = 3 gives 1 - i), so both parts are returned as signed
integers (each 0 or +-2^p).
"""
from __future__ import annotations


def expsum_z2(M, L) -> int:
    """sum_{x in {0,1}^n} (-1)^{x M x^T + L x^T}  (Eq. (Zreal)).

    M: n x n binary matrix (list of lists; need not be symmetric, may have a
    diagonal), L: list of n bits.
    """
    n = len(L)
    if n == 0:
        return 1
    pair = None
    for a in range(n):
        for b in range(a + 1, n):
            if M[a][b] != M[b][a]:
                pair = (a, b)
                break
        if pair:
            break
    if pair is None:
        # Symmetric M: the quadratic terms cancel, Q(x) = (L + diag M) x^T.
        return (1 << n) if all((L[a] + M[a][a]) % 2 == 0 for a in range(n)) else 0
    a, b = pair
    rest = [i for i in range(n) if i not in (a, b)]
    c1 = (L[a] + M[a][a]) % 2
    c2 = (L[b] + M[b][b]) % 2
    m1 = [(M[a][i] + M[i][a]) % 2 for i in rest]
    m2 = [(M[b][i] + M[i][b]) % 2 for i in rest]
    # Q'(y) = y (M_else + m1^T m2) y^T + (L_else + c1 m2 + c2 m1) y^T   (Eq. (eq5))
    Mp = [[(M[i][j] + m1[ii] * m2[jj]) % 2 for jj, j in enumerate(rest)]
          for ii, i in enumerate(rest)]
    Lp = [(L[i] + c1 * m2[ii] + c2 * m1[ii]) % 2 for ii, i in enumerate(rest)]
    # sum_{x1,x2} (-1)^{x1 x2 + mu1 x1 + mu2 x2} = 2 (-1)^{mu1 mu2}   (Eq. (identity))
    return 2 * (-1) ** (c1 * c2) * expsum_z2(Mp, Lp)


def expsum(B) -> tuple[int, int]:
    """Z(B) for B in M_n (symmetric; off-diagonal mod 2, diagonal mod 4).

    Returns (Re Z, Im Z) as integers.
    """
    n = len(B)
    # B_{aa} = 2 L_a + K_a; M upper triangle of B  (Eq. (q))
    K = [B[a][a] % 2 for a in range(n)]
    L = [(B[a][a] % 4) // 2 for a in range(n)]
    # Z2 form on n+1 variables (Eq. (Q)):
    # sum_{a<b} (M_ab + K_a K_b) x_a x_b + sum_a K_a x_a x_{n+1} + sum_a L_a x_a
    Mt = [[0] * (n + 1) for _ in range(n + 1)]
    for a in range(n):
        for b in range(a + 1, n):
            Mt[a][b] = (B[a][b] + K[a] * K[b]) % 2
        Mt[a][n] = K[a]
    re2 = expsum_z2(Mt, L + [0])
    im2 = expsum_z2(Mt, L + [1])
    assert re2 % 2 == 0 and im2 % 2 == 0
    return re2 // 2, im2 // 2  # Eq. (real)
