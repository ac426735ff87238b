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
        assert c["k_chunk"] <= 256 and c["k_chunk"] % c["stage_points"] == 0
        assert c["k_chunk"] >= 2 * c["stage_points"]


def test_candidates_are_valid_tilings():
    for path, cands in autotune.CANDIDATES.items():
        assert cands[0]["flags"] == autotune.PAIR  # the library's default first
        for c in cands:
            assert c["flags"] in (autotune.PAIR, autotune.ONE_CTA)
            assert c["tile_n"] in (128, 256) and c["stage_points"] in (32, 64)
            if c["flags"] == autotune.PAIR:
                assert c["tile_n"] == 256 and c["stage_points"] == 64


class _Pts:
    def __init__(self, n):
        self.shape = (n, 2)


def test_tune_batch_gives_each_gaussian_instance_its_class_tiling(tmp_path):
    cache = str(tmp_path / "tune.json")
    calls = []

    def timer(run):  # a fake clock: the fourth candidate (128 x 128, one CTA) wins
        calls.append(run)
        return 1.0 if len(calls) % len(autotune.CANDIDATES["tc_split16"]) == 4 else 2.0

    base = dict(origin=(0.0, 0.0), cell=10.0, h=50.0, weights=None)
    insts = [dict(base, points=_Pts(1000), nx=128, ny=128, kernel="gaussian"),
             dict(base, points=_Pts(1000), nx=128, ny=128, kernel="epanechnikov"),
             dict(base, points=_Pts(1100), nx=130, ny=120, kernel="gaussian"),
             dict(base, points=_Pts(4000), nx=2048, ny=2048, kernel=6)]
    tl = autotune.tune_batch(insts, cache_path=cache, timer=timer)
    assert tl[1] is None
    assert tl[0] == tl[2] == autotune.CANDIDATES["tc_split16"][3]
    # two classes, each timed once per candidate; the cache serves a second call
    assert len(calls) == 2 * len(autotune.CANDIDATES["tc_split16"])
    assert autotune.tune_batch(insts, cache_path=cache, timer=timer) == tl
    assert len(calls) == 2 * len(autotune.CANDIDATES["tc_split16"])


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "cache.json")
    autotune.save_cache({"k": {"opts": {"tile_n": 256}, "ms": 1.5}}, p)
    assert autotune.load_cache(p)["k"]["opts"] == {"tile_n": 256}
    assert json.load(open(p))["k"]["ms"] == 1.5
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}
