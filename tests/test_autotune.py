"""The autotuner's transaction model and cache (no GPU)."""
from paper_2007_04457_gb300 import autotune


def test_model_counts_halo_rows():
    # taller tiles re-read fewer halo rows on a big grid
    big = (513, 513, 513)
    v = {c: autotune.restriction_model(big, 4, c) for c in autotune.CONFIGS}
    assert v[2] < v[0] < v[1]
    assert all(x > 1.0 for x in v.values())
    # on a grid one tile tall the tall tile wastes nothing extra
    small = (17, 17, 17)
    assert autotune.restriction_model(small, 4, 2) <= autotune.restriction_model(small, 4, 1)


def test_tile_rows():
    assert [autotune.tile_rows(c, 3, 4) for c in autotune.CONFIGS] == [8, 4, 16]


def test_tiles_absorb_the_last_node():
    assert autotune._tiles(257, 8) == [8] * 31 + [9]
    assert autotune._tiles(17, 16) == [17]
    assert autotune._tiles(2, 8) == [2]
    assert sum(autotune._tiles(513, 64)) == 513


def test_ranked_configs_prunes_to_top():
    r = autotune.ranked_configs((257, 257, 257), 4, top=2)
    assert len(r) == 2 and r[0] == 2


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert autotune.load_cache(path) == {}
    key = autotune.cache_key("GB300", (33, 65), "f32")
    autotune.save_cache({key: {"cfg": 1, "warps": 8, "ms": 0.5}}, path)
    assert autotune.load_cache(path)[key]["warps"] == 8
