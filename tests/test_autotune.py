"""The batch autotuner on a stand-in batch (no GPU): it consumes exactly the steps it
announces, whichever candidates win, and returns the fastest shape it timed."""
import itertools

from paper_1311_2147_gb300 import autotune


class FakeBatch:
    """Step time = a fixed cost per tile value (lower is faster); counts applied steps."""

    def __init__(self, cost):
        self.cost = cost
        self.tiles = None
        self.steps = 0

    def bc_batch_set_tiles(self, tiles):
        self.tiles = list(tiles)

    def bc_batch_apply(self, lists):
        self.steps += 1
        return 0, None

    def bc_batch_last_ms(self):
        return float(sum(self.cost(i, v) for i, v in enumerate(self.tiles)))

    def last_error(self):
        return ""


def _run(cost):
    b = FakeBatch(cost)
    calls = itertools.count()
    tiles, trials = autotune.tune(b, lambda: next(calls), key=None, use_cache=False)
    return b, tiles, trials


def test_step_count_when_the_first_candidate_wins():
    # every parameter's first listed value is best, so the incumbent changes mid-list
    b, tiles, trials = _run(lambda i, v: autotune.CANDIDATES[i].index(v))
    assert b.steps == autotune.steps_needed()
    assert len(trials) == 1 + sum(len(c) - 1 for c in autotune.CANDIDATES)
    assert tiles == [c[0] for c in autotune.CANDIDATES]


def test_step_count_when_the_last_candidate_wins():
    b, tiles, trials = _run(lambda i, v: -autotune.CANDIDATES[i].index(v))
    assert b.steps == autotune.steps_needed()
    assert tiles == [c[-1] for c in autotune.CANDIDATES]
    best = min(ms for _, ms in trials)
    assert dict((tuple(t), ms) for t, ms in trials)[tuple(tiles)] == best


def test_defaults_are_candidates():
    assert len(autotune.DEFAULT) == len(autotune.CANDIDATES)
    for d, c in zip(autotune.DEFAULT, autotune.CANDIDATES):
        assert d in c
