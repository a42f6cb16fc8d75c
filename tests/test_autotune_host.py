"""Host logic of the autotuner's cache (no GPU): shape keys bucket the sample
count by powers of two, the JSON table round-trips, a missing or corrupt
file reads as empty."""
import os

import pytest

pytest.importorskip("torch")


def test_shape_key_buckets_and_cache_round_trip(tmp_path):
    from paper_2507_22128_gb300 import autotune
    k1 = autotune.shape_key(1024, 16, 4, 2, 8_000_000)
    k2 = autotune.shape_key(1024, 16, 4, 2, 8_300_000)     # same power of two
    k3 = autotune.shape_key(1024, 16, 4, 2, 17_000_000)
    k4 = autotune.shape_key(512, 16, 4, 2, 8_000_000)
    assert k1 == k2 and k1 != k3 and k1 != k4
    path = str(tmp_path / "sub" / "t.json")
    assert autotune.load(path) == {}
    autotune.save(path, {k1: {"chunk_limit": 16, "ctas_per_sm": 0, "ms": 1.0}})
    assert autotune.load(path)[k1]["chunk_limit"] == 16
    with open(path, "w") as f:
        f.write("{not json")
    assert autotune.load(path) == {}
    os.environ["RIX_AUTOTUNE_CACHE"] = path
    try:
        assert autotune.default_cache_path() == path
    finally:
        del os.environ["RIX_AUTOTUNE_CACHE"]
