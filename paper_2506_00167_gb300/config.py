"""A decoder session's configuration as JSON: the base graphs (shape and entries, each with a SHA-256),
the lifting sizes and the arithmetic (mode, iterations, early exit, offsets, quantiser), so that a run can
be repeated bit for bit from a file.  Decoding keeps no state between calls, so this is all a run needs
besides its inputs (the autotuned tiles are cached as JSON on their own)."""
from __future__ import annotations

import hashlib
import json
from dataclasses import dataclass

import numpy as np

VERSION = 1


@dataclass
class BaseGraphSpec:
    """A base graph as the session takes it: shape and (row, col, V) entries."""
    mb: int
    nb: int
    kb: int
    mc: int
    n_punct_cols: int
    row: np.ndarray
    col: np.ndarray
    V: np.ndarray


def _digest(g) -> str:
    h = hashlib.sha256()
    h.update(np.array([g.mb, g.nb, g.kb, g.mc, g.n_punct_cols], dtype=np.int64).tobytes())
    for a in (g.row, g.col, g.V):
        h.update(np.ascontiguousarray(a, dtype=np.int16).tobytes())
    return h.hexdigest()


def session_config(base_graphs, z_set, mode: str = "f32", max_iter: int = 10, early_term: bool = True,
                   offset_f32: float = 0.5, offset_lsb: int = 1, q_scale: float = 4.0, sat=None,
                   interleave: bool = True) -> dict:
    """The configuration Session(base_graphs, z_set, ...) would run with, defaults made explicit."""
    from .session import DEFAULT_SAT
    if mode not in DEFAULT_SAT:
        raise ValueError(f"unknown mode {mode!r}")
    llr_sat, msg_sat, post_sat = DEFAULT_SAT[mode] if sat is None else sat
    graphs = []
    for g in base_graphs:
        entries = np.stack([np.asarray(g.row, np.int64), np.asarray(g.col, np.int64), np.asarray(g.V, np.int64)], 1)
        graphs.append({"mb": int(g.mb), "nb": int(g.nb), "kb": int(g.kb), "mc": int(g.mc),
                       "n_punct_cols": int(g.n_punct_cols), "entries": entries.tolist(), "sha256": _digest(g)})
    return {"version": VERSION, "base_graphs": graphs, "z_set": [int(z) for z in z_set], "mode": mode,
            "max_iter": int(max_iter), "early_term": bool(early_term), "offset_f32": float(offset_f32),
            "offset_lsb": int(offset_lsb), "q_scale": float(q_scale),
            "sat": [int(llr_sat), int(msg_sat), int(post_sat)], "interleave": bool(interleave)}


def dumps(cfg: dict) -> str:
    return json.dumps(cfg, sort_keys=True)


def session_args(cfg: dict):
    """(base graphs, z_set, keyword arguments) for Session, after checking every graph's digest."""
    if cfg.get("version") != VERSION:
        raise ValueError(f"configuration version {cfg.get('version')!r}, expected {VERSION}")
    graphs = []
    for i, d in enumerate(cfg["base_graphs"]):
        e = np.asarray(d["entries"], dtype=np.int64).reshape(-1, 3)
        g = BaseGraphSpec(d["mb"], d["nb"], d["kb"], d["mc"], d["n_punct_cols"], e[:, 0].astype(np.int16),
                          e[:, 1].astype(np.int16), e[:, 2].astype(np.int16))
        if _digest(g) != d["sha256"]:
            raise ValueError(f"base graph {i}: entries do not match their SHA-256")
        graphs.append(g)
    kw = {k: cfg[k] for k in ("mode", "max_iter", "early_term", "offset_f32", "offset_lsb", "q_scale",
                              "interleave")}
    kw["sat"] = tuple(cfg["sat"])
    return graphs, list(cfg["z_set"]), kw


def loads(text: str):
    """session_args of a configuration written by dumps."""
    return session_args(json.loads(text))


def session_from_config(cfg: dict):
    """A Session (on the current CUDA device) with exactly this configuration."""
    from .session import Session
    graphs, z_set, kw = session_args(cfg)
    return Session(graphs, z_set, **kw)
