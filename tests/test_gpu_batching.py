"""Persistent uneven batching: launch plans, tiles, CUDA-graph capture, autotuner (GPU)."""
import json

import numpy as np
import pytest
import torch

from oracle import decoder as odec
from oracle import demap as odemap
from paper_2506_00167_gb300 import Graph
from paper_2506_00167_gb300.autotune import autotune, autotune_batch, tiles_from_cache
from workload import mixed

from gpu_helpers import device_inputs, session_for, to_np_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wmix():
    return mixed(n_slots=4, ues_per_slot=6, max_cb=3, seed=21)


def _decode(s, w, llr_np, dtype):
    b = s.batch(w.cbs)
    bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
    status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
    s.decode_batch(b, torch.from_numpy(llr_np.astype(dtype)).cuda(), bits, status)
    return to_np_u32(bits), status.cpu().numpy(), b.plan()


def test_plans_and_tiles_do_not_change_results(wmix):
    w = wmix
    llr_np = odemap.quantise(odemap.demap_workload(w), 4.0, 63)
    want_bits, want_status = odec.decode_workload(w, llr_np, 10, True, odec.INT8)
    seen_plans = []
    for strategy, tiles in [("mixed", None), ("per_z", None), ("mixed", "one"), ("mixed", "max")]:
        s = session_for(w, "i8")
        s.set_strategy(strategy)
        if tiles == "one":
            s.set_tiles([(b, z, 1 if z > 16 else 2) for b in range(2) for z in w.z_set])
        elif tiles == "max":
            s.set_tiles([(b, z, min(15, 512 // z) if z > 32 else 512 // z) for b in range(2) for z in w.z_set])
        bits, status, plan = _decode(s, w, llr_np, np.int8)
        assert np.array_equal(bits, want_bits), (strategy, tiles)
        assert np.array_equal(status, want_status), (strategy, tiles)
        seen_plans.append(plan)
    n_z = len(set(int(z) for z in w.cbs["Z"]))
    assert len(seen_plans[0]) == 1            # one persistent launch over every shape
    assert len(seen_plans[1]) == n_z          # one per lifting size
    assert seen_plans[0][0]["n_items"] < seen_plans[2][0]["n_items"]


def test_graph_replay_matches_direct_calls(wmix):
    w = wmix
    s = session_for(w, "i8")
    b = s.batch(w.cbs, w.tbs, w.slot_N)
    sym, mask = device_inputs(w)
    ref = s.run(b, sym, mask, b.alloc_outputs())
    out = b.alloc_outputs()
    g = Graph(s, b, sym, mask, out)
    for _ in range(2):
        for t in out.values():
            t.zero_()
        g.launch()
        torch.cuda.synchronize()
        for k in ["llr", "bits", "status", "d", "goodput_bits", "goodput_sc", "reward"]:
            assert torch.equal(out[k], ref[k]), k
    g.close()


def test_autotune_picks_a_feasible_tile_and_round_trips(tmp_path, wmix):
    w = wmix
    cache = tmp_path / "tiles.json"
    res = autotune(w.bgs, [32, 64], mode="i8", n_cb=256, max_iter=2, reps=2, cache_path=str(cache),
                   shapes=[(1, 32), (1, 64)], cands=lambda Z: [1, 2] if Z > 32 else [2, 4])
    assert len(res["tiles"]) == 2
    for t in res["tiles"]:
        assert t["G"] in (1, 2, 4) and t["us_per_cb"] > 0
    data = json.loads(cache.read_text())
    assert any("|i8" in k for k in data)
    tiles = tiles_from_cache(str(cache), w.bgs, "i8")
    assert sorted((z for _, z, _ in tiles)) == [32, 64]
    s = session_for(w, "i8")
    assert s.load_tiles(str(cache), w.bgs) == 2


def test_batch_autotuner_never_loses_to_default_and_keeps_results(tmp_path, wmix):
    """Coordinate descent on the whole batch: the tuned time is no worse than the built-in tiles', the tiles
    apply to a session, and decoding under them gives the oracle's bits."""
    w = wmix
    cache = tmp_path / "tiles.json"
    ent = autotune_batch(w.bgs, w.z_set, w.cbs, mode="i8", max_iter=2, reps=2, sweeps=1, cache_path=str(cache),
                         tag="mix", cands=lambda Z: [1, 2])
    assert ent["tuned_ms"] <= ent["default_ms"] and ent["trials"] >= 1
    assert tiles_from_cache(str(cache), w.bgs, "i8") == []          # tagged entry only
    s = session_for(w, "i8")
    assert s.load_tiles(str(cache), w.bgs, tag="mix") == len({(int(c["bg"]), int(c["Z"])) for c in w.cbs})
    llr_np = odemap.quantise(odemap.demap_workload(w), 4.0, 63)
    want_bits, want_status = odec.decode_workload(w, llr_np, 10, True, odec.INT8)
    bits, status, plan = _decode(s, w, llr_np, np.int8)
    assert len(plan) == 1
    assert np.array_equal(bits, want_bits) and np.array_equal(status, want_status)
