"""Pins for the oracle's counter-based generator (SplitMix64 in counter mode)."""
import json
import os

from oracle import rng

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64_state0.json")))


def test_mix_reproduces_published_splitmix64_outputs():
    """Output k of SplitMix64 from state 0 is mix(k G): a wrong shift, constant or
    order of the mix steps changes these published values."""
    for k, want in enumerate(GOLD["outputs"], start=1):
        assert rng.mix(k * rng.GOLDEN) == int(want, 16)


def test_counter_mode_is_the_splitmix_sequence_of_the_key():
    """rand64(seed, stream, i) is output i+1 of SplitMix64 started from state
    key(seed, stream); key is the mix of seed ^ mix(stream + G)."""
    for seed, stream in ((0, 0), (7, 3), (2 ** 64 - 1, 2 ** 41)):
        k = rng.key(seed, stream)
        assert k == rng.mix(seed ^ rng.mix(stream + rng.GOLDEN))
        state = k
        for i in range(5):
            state = (state + rng.GOLDEN) & rng.MASK64
            assert rng.rand64(seed, stream, i) == rng.mix(state)


def test_uniform_is_53_bit():
    for i in range(200):
        u = rng.uniform(3, 5, i)
        assert 0.0 <= u < 1.0
        assert u * 2 ** 53 == int(u * 2 ** 53)
        assert int(u * 2 ** 53) == rng.rand64(3, 5, i) >> 11
