"""Autotuner bookkeeping that needs no GPU: candidate tiles, cache keys, synthetic descriptors."""
import json

import numpy as np

from paper_2506_00167_gb300 import autotune as at
from workload import default_bgs


def test_candidates_respect_block_and_barrier_limits():
    for mode, cap in [("i8", 384), ("f32", 384), ("i16", 384)]:
        for Z in [16, 32, 64, 128, 256, 384]:
            c = at.candidates(Z, mode)
            assert c and all(g * Z <= cap for g in c)
            if Z > 32:
                assert max(c) <= 15
            if Z == 16:
                assert all(g % 2 == 0 for g in c)


def test_synthetic_descriptors_are_valid_shapes():
    bgs = default_bgs()
    cbs = at.synthetic_cbs(bgs[0], 0, 384, 8)
    assert np.all(cbs["E"] == 16896) and np.all(np.diff(cbs["llr_offset"]) == 46 * 384)
    assert np.all(cbs["llr_offset"] % 16 == 0)


def test_cache_round_trip_by_graph_hash(tmp_path):
    bgs = default_bgs()
    path = tmp_path / "c.json"
    data = {"GB300|i8": {"device": "GB300", "mode": "i8", "tiles": [
        {"bg": at.bg_key(bgs[1]), "Z": 64, "G": 3}, {"bg": "unknown", "Z": 32, "G": 8}]}}
    path.write_text(json.dumps(data))
    assert at.tiles_from_cache(str(path), bgs, "i8", device_name="GB300") == [(1, 64, 3)]
    assert at.tiles_from_cache(str(path), bgs, "f32", device_name="GB300") == []
    assert at.bg_key(bgs[0]) != at.bg_key(bgs[1])


def test_default_tile_matches_the_planner_caps():
    for Z, G in [(16, 16), (32, 8), (64, 4), (128, 2), (256, 1), (384, 1)]:
        assert at.default_tile(Z) == G
        assert at.default_tile(Z) * Z <= at.MAX_BLOCK


def test_tagged_cache_entries_are_separate(tmp_path):
    bgs = default_bgs()
    path = tmp_path / "c.json"
    data = {at.cache_key("GB300", "i8", "mixed"): {"tiles": [{"bg": at.bg_key(bgs[0]), "Z": 32, "G": 6}]},
            at.cache_key("GB300", "i8"): {"tiles": [{"bg": at.bg_key(bgs[0]), "Z": 32, "G": 2}]}}
    path.write_text(json.dumps(data))
    assert at.tiles_from_cache(str(path), bgs, "i8", device_name="GB300", tag="mixed") == [(0, 32, 6)]
    assert at.tiles_from_cache(str(path), bgs, "i8", device_name="GB300") == [(0, 32, 2)]
    assert at.tiles_from_cache(str(path), bgs, "i8", device_name="GB300", tag="large") == []
