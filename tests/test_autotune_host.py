"""Host logic of the autotuner (CPU): candidate enumeration, choice of the
fastest setting and the JSON cache round trip."""
import os

from paper_2308_13476_gb300 import autotune


def test_candidates_cover_the_space():
    space = {"tile_rows": [1, 2], "coarse_nodes": [300], "coarse_mode": [0, 1]}
    c = list(autotune.candidates(space))
    assert len(c) == 4
    assert {"tile_rows": 2, "coarse_nodes": 300, "coarse_mode": 1} in c


def test_best_of_picks_lowest_time_first_on_ties():
    res = [dict(a=1, ms_per_cycle=2.0), dict(a=2, ms_per_cycle=1.0), dict(a=3, ms_per_cycle=1.0)]
    assert autotune.best_of(res)["a"] == 2


def test_cache_round_trip(tmp_path):
    p = os.path.join(tmp_path, "tune.json")
    assert autotune.load_cache(p) == {}
    key = autotune.cache_key("GPU", 8, 8, 2, "mixed", "gmres3", "V", 2)
    autotune.store_cache(p, {key: {"best": {"tile_rows": 1}, "results": []}})
    assert autotune.load_cache(p)[key]["best"] == {"tile_rows": 1}
