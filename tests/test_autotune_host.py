"""Host logic of the launch-shape autotuner (no GPU): the incumbent value of a knob
stays unless another candidate is faster by more than the margin, values outside the
candidate list are not incumbents, and cached choices are applied without timing."""
import os
import tempfile

from paper_1808_00128_gb300 import autotune


class FakeSim:
    n, chi, device = 40, 1 << 16, 0

    def __init__(self, **tuning):
        self.tuning = dict(mc_chains_per_block=64, mc_stages=2, mc_lookahead=2)
        self.tuning.update(tuning)

    def set_tuning(self, name, value):
        self.tuning[name] = value

    def get_tuning(self, name):
        return self.tuning[name]

    def metropolis(self, steps, seed):
        pass


def _timer(sim, table):
    """Milliseconds as a function of the current (chains per block, stages)."""
    calls = []

    def t(fn):
        fn()
        key = (sim.get_tuning("mc_chains_per_block"), sim.get_tuning("mc_stages"))
        calls.append(key)
        return table.get(key, 10.0)
    return t, calls


def test_incumbent_kept_within_margin():
    sim = FakeSim()
    t, _ = _timer(sim, {(64, 2): 1.00, (32, 2): 0.98, (32, 1): 2.0, (64, 1): 2.0, (64, 3): 1.5, (64, 4): 1.5})
    chosen = autotune.tune(sim, chains=256, timer=t)
    assert chosen["mc_chains_per_block"][0] == 64     # 2% faster is within the margin
    assert chosen["mc_stages"][0] == 2


def test_clearly_faster_candidate_wins():
    sim = FakeSim()
    t, _ = _timer(sim, {(64, 2): 1.00, (32, 2): 0.90, (32, 3): 0.80, (32, 1): 2.0, (32, 4): 0.85})
    chosen = autotune.tune(sim, chains=256, timer=t)
    assert chosen["mc_chains_per_block"][0] == 32
    assert chosen["mc_stages"][0] == 3
    assert sim.get_tuning("mc_stages") == 3


def test_value_outside_candidates_is_no_incumbent():
    sim = FakeSim(mc_chains_per_block=7)
    t, calls = _timer(sim, {(32, 2): 1.0, (64, 2): 1.01, (7, 2): 0.1})
    chosen = autotune.tune(sim, chains=256, timer=t)
    assert chosen["mc_chains_per_block"][0] in autotune.CANDIDATES["mc_chains_per_block"]
    assert (7, 2) not in calls


def test_cached_choice_applied_without_timing():
    sim = FakeSim()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.json")
        t, _ = _timer(sim, {(64, 2): 1.0, (32, 2): 0.5, (32, 4): 0.4})
        first = autotune.tune(sim, chains=256, cache_path=path, timer=t)
        sim2 = FakeSim()
        t2, calls2 = _timer(sim2, {})
        second = autotune.tune(sim2, chains=256, cache_path=path, timer=t2)
        assert calls2 == []
        assert {k: v[0] for k, v in second.items()} == {k: v[0] for k, v in first.items()}
        assert sim2.get_tuning("mc_chains_per_block") == 32 and sim2.get_tuning("mc_stages") == 4
