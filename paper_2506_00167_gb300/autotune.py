"""Autotuner for the decoder's work-item tiles.

A tile is G: how many code blocks of one (base graph, Z) shape a thread block
decodes side by side (G groups of Z threads).  Larger G means more warps per
block and fewer block-level hand-offs; smaller G means less shared memory per
block and therefore more resident blocks.  The best G depends on the shape,
the mode, the GPU and -- because a mixed batch is one persistent launch whose
block size is the largest G * Z of its shapes -- on the other shapes in the
batch.  So it is measured:

* ``autotune`` times each shape alone, on a synthetic batch large enough to
  fill the GPU, for every feasible G and keeps the fastest;
* ``autotune_batch`` tunes the tiles of every shape of a given batch
  together, by coordinate descent on the decode time of the whole batch,
  starting from the built-in tiles and keeping a change only when it gains.

Both time ``decode_batch`` with a fixed iteration count and early termination
off on random LLRs (the per-iteration cost does not depend on the values).
Results are cached as JSON keyed by the GPU name, the mode and an optional
workload tag, with each tile keyed by a hash of its base graph, and applied to
a session with ``Session.load_tiles``.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import abi

MAX_BLOCK = 384  # two decoder blocks share an SM's registers


def candidates(Z: int, mode: str = "i8") -> list:
    """Feasible tiles G for lifting size Z (G * Z <= 384; one named barrier per group for Z > 32).
    The bound is the same for every mode; `mode` is accepted for symmetry with the tuner."""
    del mode
    if Z > 32:
        return list(range(1, min(15, MAX_BLOCK // Z) + 1))
    if Z == 32:
        return list(range(1, MAX_BLOCK // Z + 1))
    return list(range(2, MAX_BLOCK // Z + 1, 2))  # Z = 16: groups come in half-warp pairs


def bg_key(g) -> str:
    h = hashlib.sha256()
    for v in (g.mb, g.nb, g.kb, g.mc, g.n_punct_cols):
        h.update(int(v).to_bytes(4, "little", signed=True))
    for arr in (g.row, g.col, g.V):
        h.update(np.ascontiguousarray(arr, dtype=np.int16).tobytes())
    return h.hexdigest()[:16]


def synthetic_cbs(g, bg_index: int, Z: int, n_cb: int, rate: float = 0.5, Qm: int = 2) -> np.ndarray:
    """Descriptors of n_cb code blocks of one shape at the given rate, LLRs packed back to back."""
    K = g.kb * Z
    t0 = g.n_punct_cols * Z
    E = Qm * int(round(K / (rate * Qm)))
    E = min(E, (g.nb * Z - t0) // Qm * Qm)
    cols = -(-(E + t0) // Z)
    m_eff = min(g.mb, max(g.mc, cols - g.kb))
    n_llr = (g.kb + m_eff) * Z
    cbs = np.zeros(n_cb, dtype=abi.CB_NP)
    cbs["bg"] = bg_index
    cbs["Z"] = Z
    cbs["Qm"] = Qm
    cbs["E"] = E
    cbs["re_offset"] = np.arange(n_cb) * (E // Qm)
    cbs["mask_word_offset"] = np.arange(n_cb) * (-(-(E // Qm) // 32))
    cbs["llr_offset"] = np.arange(n_cb) * n_llr
    cbs["bits_word_offset"] = np.arange(n_cb) * (K // 32)
    cbs["inv_sigma2"] = 1.0
    return cbs


def default_tile(Z: int) -> int:
    """The library's built-in tile (as the planner applies it: G * Z <= 384, even G for Z = 16)."""
    G = max(1, 256 // Z)
    if Z > 32:
        G = min(G, 15)
    G = min(G, max(1, MAX_BLOCK // Z))
    if Z == 16 and G > 1 and G % 2:
        G -= 1
    return G


def _random_llr(n: int, mode: str):
    import torch

    from .session import DEFAULT_SAT, LLR_TORCH
    if mode == "f32":
        return torch.randn(n, device="cuda", dtype=torch.float32) * 4.0
    lim = DEFAULT_SAT[mode][0]
    return torch.randint(-lim, lim + 1, (n,), device="cuda", dtype=torch.int32).to(LLR_TORCH[mode])


def _time_decode(base_graphs, z_set, mode, max_iter, tiles, cbs, reps, llr_cache):
    """Mean decode_batch time (ms) of the batch `cbs` under the given tiles, or None if it does not plan."""
    import torch

    from .session import DEFAULT_SAT, Session
    s = Session(base_graphs, z_set, mode=mode, max_iter=max_iter, early_term=False,
                sat=DEFAULT_SAT[mode] if mode != "f32" else None)
    try:
        s.set_tiles(tiles)
        bt = s.batch(cbs)
    except abi.LdpcError:
        s.close()
        return None
    n = bt.info.llr_elems
    if llr_cache.get("n") != n:
        llr_cache["n"], llr_cache["llr"] = n, _random_llr(n, mode)
    llr = llr_cache["llr"]
    bits = torch.empty(bt.info.bits_words, dtype=torch.int32, device="cuda")
    status = torch.empty(bt.n_cb, dtype=torch.int32, device="cuda")
    for _ in range(2):
        s.decode_batch(bt, llr, bits, status)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        s.decode_batch(bt, llr, bits, status)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del bt
    s.close()
    return ms


def _write_cache(cache_path, key, entry):
    merged = {}
    if os.path.exists(cache_path):
        with open(cache_path) as f:
            merged = json.load(f)
    prev = {(t["bg"], t["Z"]): t for t in merged.get(key, {}).get("tiles", [])}
    for t in entry["tiles"]:
        prev[(t["bg"], t["Z"])] = t
    merged[key] = dict(entry, tiles=list(prev.values()))
    with open(cache_path, "w") as f:
        json.dump(merged, f, indent=1, sort_keys=True)


def cache_key(device: str, mode: str, tag: str | None = None) -> str:
    return f"{device}|{mode}" + (f"|{tag}" if tag else "")


def autotune_batch(base_graphs, z_set, cbs, mode: str = "i8", max_iter: int = 3, reps: int = 3,
                   sweeps: int = 2, min_gain: float = 0.01, cache_path: str | None = None,
                   tag: str | None = None, cands=None) -> dict:
    """Tiles for every shape of the batch `cbs`, tuned together on the batch's decode time."""
    import torch

    dev_name = torch.cuda.get_device_name()
    shapes = sorted({(int(c["bg"]), int(c["Z"])) for c in cbs})
    tiles = {sh: default_tile(sh[1]) for sh in shapes}
    llr_cache = {}

    def measure(t):
        return _time_decode(base_graphs, z_set, mode, max_iter, [(b, z, g) for (b, z), g in t.items()], cbs, reps,
                            llr_cache)

    base_ms = best = measure(tiles)
    if best is None:
        raise RuntimeError("the batch does not plan with the built-in tiles")
    trials = 1
    for _ in range(sweeps):
        improved = False
        for sh in shapes:
            for G in (cands(sh[1]) if cands else candidates(sh[1], mode)):
                if G == tiles[sh]:
                    continue
                trial = dict(tiles)
                trial[sh] = G
                ms = measure(trial)
                trials += 1
                if ms is not None and ms < best * (1.0 - min_gain):
                    best, tiles, improved = ms, trial, True
        if not improved:
            break
    entry = {"device": dev_name, "mode": mode, "objective": "whole-batch decode time", "tag": tag,
             "default_ms": base_ms, "tuned_ms": best, "trials": trials,
             "tiles": [{"bg": bg_key(base_graphs[b]), "bg_shape": [base_graphs[b].mb, base_graphs[b].nb,
                                                                 base_graphs[b].kb], "Z": z, "G": g}
                       for (b, z), g in tiles.items()]}
    if cache_path:
        _write_cache(cache_path, cache_key(dev_name, mode, tag), entry)
    return entry


def autotune(base_graphs, z_set, mode: str = "i8", n_cb: int | None = None, max_iter: int = 3, reps: int = 5,
             cache_path: str | None = None, shapes=None, cands=None, tag: str | None = None) -> dict:
    """Time every feasible tile for each (base graph, Z) alone; returns (and optionally caches) the results.
    Each shape's synthetic batch holds n_cb code blocks, by default as many lifted variables as 2048
    blocks at Z = 384, so every tile fills the GPU."""
    import torch

    from .session import DEFAULT_SAT, LLR_TORCH, Session

    dev_name = torch.cuda.get_device_name()
    result = {"device": dev_name, "mode": mode, "tiles": []}
    todo = shapes if shapes is not None else [(b, Z) for b in range(len(base_graphs)) for Z in z_set]
    for b, Z in todo:
        g = base_graphs[b]
        if (g.kb * Z) % 32:
            continue
        nb = n_cb if n_cb else max(64, 2048 * 384 // Z)
        cbs = synthetic_cbs(g, b, Z, nb)
        timings = {}
        for G in (cands(Z) if cands else candidates(Z, mode)):
            s = Session(base_graphs, [Z], mode=mode, max_iter=max_iter, early_term=False, sat=DEFAULT_SAT[mode]
                        if mode != "f32" else None)
            s.set_tiles([(b, Z, G)])
            try:
                bt = s.batch(cbs)
            except abi.LdpcError:
                continue
            plan = bt.plan()
            if any(p["global_messages"] for p in plan):
                pass  # still valid: the tile decides the layout of the global-message variant too
            n = bt.info.llr_elems
            if mode == "f32":
                llr = torch.randn(n, device="cuda", dtype=torch.float32) * 4.0
            else:
                lim = DEFAULT_SAT[mode][0]
                llr = torch.randint(-lim, lim + 1, (n,), device="cuda", dtype=torch.int32).to(LLR_TORCH[mode])
            bits = torch.empty(bt.info.bits_words, dtype=torch.int32, device="cuda")
            status = torch.empty(bt.n_cb, dtype=torch.int32, device="cuda")
            for _ in range(2):
                s.decode_batch(bt, llr, bits, status)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                s.decode_batch(bt, llr, bits, status)
            e1.record()
            torch.cuda.synchronize()
            timings[G] = e0.elapsed_time(e1) * 1e3 / reps / nb
            del bt, s
        if not timings:
            continue
        best = min(timings, key=timings.get)
        result["tiles"].append({"bg": bg_key(g), "bg_shape": [g.mb, g.nb, g.kb], "Z": Z, "G": best,
                                "us_per_cb": timings[best], "all_us_per_cb": {str(k): v for k, v in timings.items()}})
    if cache_path:
        _write_cache(cache_path, cache_key(dev_name, mode, tag), dict(result, objective="per-shape time"))
    return result


def tiles_from_cache(path: str, base_graphs, mode: str, device_name: str | None = None,
                     tag: str | None = None) -> list:
    """(bg index, Z, G) triples from a cache file for this GPU, mode and workload tag (empty if none)."""
    if not os.path.exists(path):
        return []
    with open(path) as f:
        data = json.load(f)
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name() if torch.cuda.is_available() else ""
    entry = data.get(cache_key(device_name, mode, tag))
    if not entry:
        return []
    keys = {bg_key(g): i for i, g in enumerate(base_graphs)}
    out = []
    for t in entry["tiles"]:
        if t["bg"] in keys:
            out.append((keys[t["bg"]], int(t["Z"]), int(t["G"])))
    return out
