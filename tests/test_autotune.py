"""Autotuner cache and selection logic (CPU, with a fake timer)."""
import json

import pytest

from paper_2004_13653_gb300 import autotune


def test_class_key_buckets():
    a = autotune.class_key("tc_split16", "gaussian", 4096, 4096, 20_000_000, 100.0, 24.4)
    b = autotune.class_key("tc_split16", "gaussian", 4000, 4100, 19_000_000, 98.0, 24.4)
    c = autotune.class_key("tc_split16", "gaussian", 1024, 4096, 20_000_000, 100.0, 24.4)
    assert a == b and a != c


def test_pick_prefers_fastest_then_first():
    assert autotune.pick([({"a": 1}, 3.0), ({"a": 2}, 1.0), ({"a": 3}, 1.0)]) == ({"a": 2}, 1.0)


def test_split_candidates_respect_accuracy_budget():
    for c in autotune.CANDIDATES["tc_split16"]:
        assert c["k_chunk"] <= 512 and c["k_chunk"] % c["stage_points"] == 0
        assert c["k_chunk"] >= 2 * c["stage_points"]


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "cache.json")
    autotune.save_cache({"k": {"opts": {"tile_n": 256}, "ms": 1.5}}, p)
    assert autotune.load_cache(p)["k"]["opts"] == {"tile_n": 256}
    assert json.load(open(p))["k"]["ms"] == 1.5
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}
