"""Host logic of the autotuner: the cache key and the JSON cache."""
from paper_2512_05516_gb300 import autotune


def test_signature_groups_similar_workloads():
    a = autotune.signature("GB300", 1_072_476, 10_648, 2000, {"v": "fp16"}, 5)
    b = autotune.signature("GB300", 1_072_476, 10_648, 2047, {"v": "fp16"}, 5)
    c = autotune.signature("GB300", 1_072_476, 10_648, 2048, {"v": "fp16"}, 5)
    d = autotune.signature("GB300", 1_072_476, 10_648, 2000, {"v": "bf16"}, 5)
    assert a == b                       # peak occupancy bucketed by powers of two
    assert a != c
    assert a != d                       # storage formats are part of the key
    assert "newton=5" in a and "GB300" in a


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "cache.json")
    assert autotune.load_cache(path) == {}
    entry = {"tuning": {"block_threads": 64, "stage_density": 768}, "ms": {"density": 1.0, "force": 2.0}}
    autotune.save_cache(path, {"k": entry})
    assert autotune.load_cache(path) == {"k": entry}
    with open(path, "w") as f:
        f.write("not json")
    assert autotune.load_cache(path) == {}


def test_search_space_is_valid():
    for bt in autotune.SPACE["block_threads"]:
        assert bt % 32 == 0 and 32 <= bt <= 256
    assert set(autotune.SPACE["subcells"]) <= {1, 2}
    assert set(autotune.SPACE["item_order"]) == {0, 1}
    assert min(autotune.SPACE["stage_density"]) >= 32 and min(autotune.SPACE["stage_force"]) >= 32
