"""The autotuner's search and cache, against a fake runtime whose step cost
is a known function of the setting (no device)."""
import math

from paper_2406_18109_gb300 import autotune
from paper_2406_18109_gb300.binding import DfsError


class FakeRuntime:
    def __init__(self, cost, fallback=lambda cfg: False, fails=lambda cfg: False):
        self.tile, self.block, self.unroll, self.ctas_per_sm = 512, 256, 2, 0
        self.tile_max = 16384
        self.rows = 16
        self.cost, self.fallback, self.fails = cost, fallback, fails
        self.ms = 0.0
        self.fallbacks = 0
        self.steps = 0

    def cfg(self):
        return autotune.current(self, autotune.PARAMS)

    def set_tiling(self, tile, rows=None, tile_max=None):
        self.tile, self.rows = tile, rows
        if tile_max is not None:
            self.tile_max = tile_max

    def set_launch(self, block, unroll, ctas_per_sm=0):
        self.block, self.unroll, self.ctas_per_sm = block, unroll, ctas_per_sm

    def step(self):
        if self.fails(self.cfg()):
            raise DfsError(-3, "cannot be resident")
        self.steps += 1
        self.ms += self.cost(self.cfg())
        if self.fallback(self.cfg()):
            self.fallbacks += 1

    def sync(self):
        pass

    def sync_quiet(self):
        pass

    def stats(self):
        return {"kernel_times": {"k": {"ms": self.ms, "launches": self.steps}}, "batch_fallbacks": self.fallbacks}


def separable(cfg):
    # optimum at tile 1024, block 128, unroll 4, ctas_per_sm 2
    return (abs(math.log2(cfg["tile"] / 1024)) + abs(math.log2(cfg["block"] / 128)) +
            abs(cfg["unroll"] - 4) * 0.5 + abs(cfg["ctas_per_sm"] - 2) * 0.25 + 1.0)


def test_coordinate_descent_finds_the_separable_optimum():
    rt = FakeRuntime(separable)
    best, trials = autotune.tune(rt, rt.step)
    assert best == {"tile": 1024, "block": 128, "unroll": 4, "ctas_per_sm": 2}
    assert autotune.current(rt) == best
    assert autotune.current(rt) == best
    assert len(trials) == 1 + 3 + 2 + 2 + 2     # start, then every other value of each parameter
    for cfg, ms in trials:
        assert abs(ms - separable(cfg)) < 1e-12


def test_fallbacks_and_failures_are_never_chosen():
    rt = FakeRuntime(separable, fallback=lambda c: c["tile"] == 1024, fails=lambda c: c["block"] == 128)
    best, trials = autotune.tune(rt, rt.step)
    assert best["tile"] != 1024 and best["block"] != 128
    assert any(math.isinf(ms) for _, ms in trials)


def test_cache_reuses_the_choice(tmp_path):
    path = str(tmp_path / "tune.json")
    rt = FakeRuntime(separable)
    best, _ = autotune.tune(rt, rt.step, key="w1", cache_path=path, gpu="g")
    rt2 = FakeRuntime(lambda cfg: 1.0)
    best2, trials2 = autotune.tune(rt2, rt2.step, key="w1", cache_path=path, gpu="g")
    assert best2 == best and rt2.steps == 0 and autotune.current(rt2) == best
    assert len(trials2) == len(_)
    # another workload key or GPU is tuned afresh
    rt3 = FakeRuntime(lambda cfg: 1.0)
    autotune.tune(rt3, rt3.step, key="w1", cache_path=path, gpu="other")
    assert rt3.steps > 0


def test_subset_space_and_tile_policy_cap():
    rt = FakeRuntime(lambda cfg: abs(math.log2(cfg["tile_max"] / 4096)) + (cfg["block"] != 128))
    rt.tile = None
    best, trials = autotune.tune(rt, lambda: rt.step(), space={"tile_max": [1024, 2048, 4096, 8192],
                                                               "block": [128, 256]})
    assert best == {"tile_max": 4096, "block": 128} and len(trials) == 1 + 4 + 1
    assert rt.tile is None and rt.tile_max == 4096


def test_rows_parameter():
    rt = FakeRuntime(lambda cfg: abs(cfg["rows"] - 32) + (cfg["unroll"] != 8))
    best, _ = autotune.tune(rt, rt.step, space={"rows": [8, 16, 32, 64], "unroll": [4, 8]})
    assert best == {"rows": 32, "unroll": 8} and rt.rows == 32


def test_ties_within_the_margin_keep_the_starting_setting():
    # every other setting is at most 1.5 % faster than the start: noise
    start = {"tile": 512, "block": 256, "unroll": 2, "ctas_per_sm": 0}
    rt = FakeRuntime(lambda cfg: 1.0 if cfg == start else 0.985 + 0.001 * cfg["unroll"] / 4)
    best, trials = autotune.tune(rt, rt.step)
    assert best == start and autotune.current(rt) == start
    # a clear win (3 %) still replaces it, and a zero margin takes any gain
    rt = FakeRuntime(lambda cfg: 0.97 if cfg["block"] == 128 else 1.0)
    assert autotune.tune(rt, rt.step)[0]["block"] == 128
    rt = FakeRuntime(lambda cfg: 1.0 if cfg == start else 0.995)
    assert autotune.tune(rt, rt.step, margin=0.0)[0] != start
