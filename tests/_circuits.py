"""Small random gate lists for the oracle pins (test helper)."""
import random


def rand_clifford(n, m, rng: random.Random, proj=False):
    ops = []
    for _ in range(m):
        k = rng.randrange(6 if proj else 5)
        if k == 0:
            ops.append(("H", rng.randrange(n)))
        elif k == 1:
            ops.append(("S", rng.randrange(n)))
        elif k in (2, 3) and n > 1:
            a, b = rng.sample(range(n), 2)
            ops.append(("CX" if k == 2 else "CZ", a, b))
        elif k == 4:
            ops.append((rng.choice(["Z", "SDG", "X"]), rng.randrange(n)))
        elif k == 5:
            ops.append((rng.choice(["P0", "P1"]), rng.randrange(n)))
        else:
            ops.append(("H", rng.randrange(n)))
    return ops
