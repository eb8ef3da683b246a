"""Autotuner for the decoder's work-item tiles.

A tile is G: how many code blocks of one (base graph, Z) shape a thread block
decodes side by side (G groups of Z threads).  Larger G means more warps per
block and fewer block-level hand-offs; smaller G means less shared memory per
block and therefore more resident blocks.  The best G depends on the shape,
the mode and the GPU, so it is measured: for each shape the tuner times
``decode_batch`` on a synthetic batch for every feasible G (fixed iteration
count, early termination off, random LLRs on the device -- the per-iteration
cost does not depend on the values) and keeps the fastest.  Results are cached
as JSON keyed by the GPU name, the mode and a hash of the base graph, and
applied to a session with ``Session.load_tiles``.
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


def autotune(base_graphs, z_set, mode: str = "i8", n_cb: int = 1024, max_iter: int = 3, reps: int = 5,
             cache_path: str | None = None, shapes=None, cands=None) -> dict:
    """Time every feasible tile for each (base graph, Z); returns (and optionally caches) the results."""
    import torch

    from .session import DEFAULT_SAT, LLR_TORCH, Session

    dev_name = torch.cuda.get_device_name()
    result = {"device": dev_name, "mode": mode, "tiles": []}
    todo = shapes if shapes is not None else [(b, Z) for b in range(len(base_graphs)) for Z in z_set]
    for b, Z in todo:
        g = base_graphs[b]
        if (g.kb * Z) % 32:
            continue
        cbs = synthetic_cbs(g, b, Z, n_cb)
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
            timings[G] = e0.elapsed_time(e1) * 1e3 / reps / n_cb
            del bt, s
        if not timings:
            continue
        best = min(timings, key=timings.get)
        result["tiles"].append({"bg": bg_key(g), "bg_shape": [g.mb, g.nb, g.kb], "Z": Z, "G": best,
                                "us_per_cb": timings[best], "all_us_per_cb": {str(k): v for k, v in timings.items()}})
    if cache_path:
        merged = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                merged = json.load(f)
        key = f"{dev_name}|{mode}"
        prev = {(t["bg"], t["Z"]): t for t in merged.get(key, {}).get("tiles", [])}
        for t in result["tiles"]:
            prev[(t["bg"], t["Z"])] = t
        merged[key] = {"device": dev_name, "mode": mode, "tiles": list(prev.values())}
        with open(cache_path, "w") as f:
            json.dump(merged, f, indent=1, sort_keys=True)
    return result


def tiles_from_cache(path: str, base_graphs, mode: str, device_name: str | None = None) -> list:
    """(bg index, Z, G) triples from a cache file for this GPU and mode (empty if none match)."""
    if not os.path.exists(path):
        return []
    with open(path) as f:
        data = json.load(f)
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name() if torch.cuda.is_available() else ""
    entry = data.get(f"{device_name}|{mode}")
    if not entry:
        return []
    keys = {bg_key(g): i for i, g in enumerate(base_graphs)}
    out = []
    for t in entry["tiles"]:
        if t["bg"] in keys:
            out.append((keys[t["bg"]], int(t["Z"]), int(t["G"])))
    return out
