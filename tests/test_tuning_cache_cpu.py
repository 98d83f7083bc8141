"""Autotuner cache keys and file round trip (host logic, no GPU)."""
from paper_2110_11398_gb300.nearfield import load_tuning_cache, save_tuning_cache, tuning_cache_key


def test_key_buckets_occupancy():
    k1 = tuning_cache_key("GB300", 2, "fp32", "plummer", 129, 134217728, 129 ** 3, 271034)
    k2 = tuning_cache_key("GB300", 2, "fp32", "plummer", 129, 134000000, 129 ** 3, 260000)
    k3 = tuning_cache_key("GB300", 2, "fp32", "plummer", 129, 134217728, 129 ** 3, 78)
    assert k1 == k2                 # same buckets
    assert k1 != k3                 # clustered vs uniform
    assert "spline" in tuning_cache_key("GB300", 2, "fp32", "spline", 65, 10, 10, 1)
    many = tuning_cache_key("GB300", 2, "fp32", "plummer", [16] * 64, 10, 10, 1)
    assert "64boxes" in many


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "tune.json")
    assert load_tuning_cache(p) == {}
    save_tuning_cache(p, {"a": {"sinks_per_lane": 4, "warps_per_block": 4}})
    assert load_tuning_cache(p)["a"]["sinks_per_lane"] == 4
    (tmp_path / "bad.json").write_text("{not json")
    assert load_tuning_cache(str(tmp_path / "bad.json")) == {}
