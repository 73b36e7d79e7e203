"""Autotuner logic without a GPU: grid search picks the fastest setting,
leaves it applied, and the JSON cache round-trips."""
import os

from paper_2308_16317_gb300 import autotune


def test_search_picks_fastest_and_applies_it(tmp_path):
    state = {}
    cost = {(1, 128): 9.0, (1, 256): 7.0, (2, 128): 5.0, (2, 256): 6.0, (4, 128): 8.0, (4, 256): 4.5,
            (8, 128): 10.0, (8, 256): 11.0}

    def set_knob(k, v):
        state[k] = v

    def run():
        # a cost with its minimum at run_tiles 32 and clusters of 2 CTAs
        return cost[(state[0], state[1])] + abs(state[3] - 32) / 64.0 + (state[7] - 2) / 8.0

    best, results = autotune.search(run, set_knob)
    assert best == {"bucket_sites": 4, "tile_n": 256, "run_tiles": 32, "cluster_ctas": 2}
    assert state == {0: 4, 1: 256, 3: 32, 7: 2}
    assert len(results) == 4 * 2 * 3 * 2
    path = os.path.join(tmp_path, "tune.json")
    key = autotune.cache_key("GB300", 1, 3, 2160, 64)
    autotune.save(path, key, best, results)
    state.clear()
    assert autotune.apply(path, key, set_knob)
    assert state == {0: 4, 1: 256, 3: 32, 7: 2}
    assert not autotune.apply(path, "other", set_knob)
