"""Counter-based random draws (oracle copy; test infrastructure only).

The generator is the SplitMix64 output function (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), used in
counter mode:

    mix(z)  = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
              z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31   (mod 2^64)
    key(seed, stream)        = mix(seed ^ mix(stream + GOLDEN))
    rand64(seed, stream, i)  = mix(key(seed, stream) + (i + 1) * GOLDEN)

with GOLDEN = 0x9E3779B97F4A7C15.  A uniform double in [0, 1) is
(rand64 >> 11) * 2^-53.  The CUDA library implements the same definition on
its own; the two share no code.
"""

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def mix(z: int) -> int:
    z &= MASK64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & MASK64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & MASK64
    z ^= z >> 31
    return z


def key(seed: int, stream: int) -> int:
    return mix((seed & MASK64) ^ mix(stream + GOLDEN))


def rand64(seed: int, stream: int, i: int) -> int:
    return mix(key(seed, stream) + (i + 1) * GOLDEN)


def uniform(seed: int, stream: int, i: int) -> float:
    return (rand64(seed, stream, i) >> 11) * (2.0 ** -53)
