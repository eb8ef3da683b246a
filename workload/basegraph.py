"""Seeded NR-style quasi-cyclic base matrices.

Input generation only.  The paper runs LDPC coding through a toolbox and
publishes no code parameters (Sec. III-B; Sec. VI-A "Tx Signal Processing"), so
the base matrices are generated from a seed rather than taken from any
standard table.  Construction (one ``BaseGraph`` per shape):

* columns ``[0, kb)`` carry information, ``[kb, kb+mc)`` core parity and
  ``[kb+mc, nb)`` extension parity;
* core rows ``r < mc``: each information column is present with probability
  ``p_core``; columns 0 and 1 are forced present in every core row of the
  BG1- and BG2-shaped matrices;
* dual-diagonal core parity: column ``kb`` has entries in rows 0,
  ``r_mid = mc // 2`` and ``mc - 1`` with raw shifts (1, 0, 1); column
  ``kb + i`` (i >= 1) has entries in rows ``i - 1`` and ``i`` with shift 0;
* extension rows ``r >= mc``: shift-0 identity on column ``kb + r``; column 0
  and column 1 each present with probability 0.7 (redrawn if neither); the
  remaining entries are distinct columns drawn uniformly from ``[2, kb+mc)``;
  the row degree is uniform in ``deg_ext``;
* every information column has degree >= 2; if the drawn matrix violates
  this, the core rows are drawn again;
* non-fixed raw shifts ``V`` are uniform in ``[0, 383]``; the lifted shift is
  ``V mod Z``; row ``k`` of a block with shift ``s`` connects to column
  ``(k + s) mod Z``.

Each base row holds at most one entry per column, so every lifted block is a
permutation and no variable is touched twice inside one layer.
"""
from __future__ import annotations

import hashlib
import json
from dataclasses import dataclass, field

import numpy as np

from .rng import SplitMix64

V_RANGE = 384  # raw shifts are drawn in [0, 384) and reduced mod Z


@dataclass(frozen=True)
class BaseGraph:
    name: str
    mb: int            # rows
    nb: int            # columns
    kb: int            # information columns
    mc: int            # core rows
    n_punct_cols: int  # leading information columns never transmitted (2 for NR-style shapes)
    row: np.ndarray = field(repr=False)   # int16, edges in row-major (row, col) order
    col: np.ndarray = field(repr=False)   # int16
    V: np.ndarray = field(repr=False)     # int16 raw shift in [0, 383]

    @property
    def n_edges(self) -> int:
        return int(self.row.size)

    def row_edges(self, r: int):
        """(cols, raw shifts) of base row ``r`` in ascending column order."""
        sel = self.row == r
        return self.col[sel].astype(np.int64), self.V[sel].astype(np.int64)

    def row_degrees(self) -> np.ndarray:
        return np.bincount(self.row.astype(np.int64), minlength=self.mb)

    def dense(self) -> np.ndarray:
        """mb x nb matrix of raw shifts, -1 where the block is zero."""
        m = -np.ones((self.mb, self.nb), dtype=np.int64)
        m[self.row, self.col] = self.V
        return m

    def sha256(self) -> str:
        payload = json.dumps({
            "name": self.name, "mb": self.mb, "nb": self.nb, "kb": self.kb,
            "mc": self.mc, "n_punct_cols": self.n_punct_cols,
            "row": self.row.tolist(), "col": self.col.tolist(), "V": self.V.tolist(),
        }, sort_keys=True).encode()
        return hashlib.sha256(payload).hexdigest()

    # ---- rate-matching geometry (shared by descriptors and the Tx chain) ----
    def t0(self, Z: int) -> int:
        """First transmitted codeword position."""
        return self.n_punct_cols * Z

    def ncb(self, Z: int) -> int:
        """Length of the circular buffer: the positions [t0, nb*Z)."""
        return self.nb * Z - self.t0(Z)

    def k0(self, Z: int, rv: int) -> int:
        """Start of redundancy version rv in the circular buffer: NR's table (3GPP TS 38.212,
        rate matching) for buffers of 66 Z and 50 Z positions, the sizes of its two base graphs;
        other graphs send redundancy version 0 only."""
        if rv == 0:
            return 0
        table = {66: (0, 17, 33, 56), 50: (0, 13, 25, 43)}
        n = self.nb - self.n_punct_cols
        if n not in table or not 0 <= rv <= 3:
            raise ValueError("redundancy versions 1-3 need a buffer of 66 Z or 50 Z positions")
        return table[n][rv] * Z

    def m_eff(self, Z: int, E: int, rv: int = 0) -> int:
        """Rows decoded for a code block that sends E bits from buffer position k0(rv).

        Columns beyond the last position sent are never transmitted (a
        transmission that wraps the buffer reaches all of them); an extension
        row whose own parity column is one of them only ever sends 0 to its
        other variables, so it is dropped.  Core rows are always kept.
        """
        k0 = self.k0(Z, rv)
        last = self.ncb(Z) if k0 + E > self.ncb(Z) else k0 + E
        cols = -(-(last + self.t0(Z)) // Z)
        return min(self.mb, max(self.mc, cols - self.kb))

    def n_eff(self, Z: int, E: int, rv: int = 0) -> int:
        return self.kb + self.m_eff(Z, E, rv)

    def peels_to_information(self, Z: int, E: int, rv: int = 0) -> bool:
        """Whether the rate-matched code can recover every information bit at all: erasure peeling on the
        lifted decoded rows (the noiseless limit of message passing), with the never-sent positions --
        the punctured leading columns and the buffer positions this transmission does not reach --
        erased.  A check with exactly one erased variable recovers it; peeling repeats until nothing
        changes.  False means some information bits stay erased at any SNR (for example, when every
        decoded row holds both punctured columns)."""
        m = self.m_eff(Z, E, rv)
        n = self.kb + m
        t0, ncb, k0 = self.t0(Z), self.ncb(Z), self.k0(Z, rv)
        known = np.zeros(n * Z, dtype=bool)
        e = np.arange(min(E, ncb))
        pos = t0 + (k0 + e) % ncb
        known[pos[pos < n * Z]] = True
        lanes = np.arange(Z)
        rows = [(c.astype(np.int64) * Z, v.astype(np.int64) % Z)
                for c, v in (self.row_edges(r) for r in range(m))]
        changed = True
        while changed and not known[:self.kb * Z].all():
            changed = False
            for base, shift in rows:
                idx = base[:, None] + (lanes[None, :] + shift[:, None]) % Z   # (edges, lanes)
                unk = ~known[idx]
                one = unk.sum(axis=0) == 1
                if one.any():
                    known[idx[:, one][unk[:, one]]] = True
                    changed = True
        return bool(known[:self.kb * Z].all())


SHAPES = {
    # name: (mb, nb, kb, mc, n_punct_cols, p_core, force01, deg_ext)
    "bg1": (46, 68, 22, 4, 2, 0.85, True, (3, 8)),
    "bg2": (42, 52, 10, 4, 2, 0.80, True, (3, 5)),
    "tiny": (8, 16, 8, 8, 0, 0.50, False, (0, 0)),
}

DEFAULT_SEEDS = {"tiny": 0, "bg1": 1, "bg2": 2}


def make_base_graph(name: str, seed: int | None = None) -> BaseGraph:
    mb, nb, kb, mc, npc, p_core, force01, (dlo, dhi) = SHAPES[name]
    rng = SplitMix64(DEFAULT_SEEDS[name] if seed is None else seed)
    r_mid = mc // 2

    def core_rows():
        rows = []
        for r in range(mc):
            ents = {}
            for j in range(kb):
                present = (force01 and j < 2) or rng.bernoulli(p_core)
                if present:
                    ents[j] = rng.below(V_RANGE)
            rows.append(ents)
        # dual-diagonal core parity
        rows[0][kb] = 1
        rows[r_mid][kb] = 0
        rows[mc - 1][kb] = 1
        for i in range(1, mc):
            rows[i - 1][kb + i] = 0
            rows[i][kb + i] = 0
        return rows

    def ext_rows():
        rows = []
        for r in range(mc, mb):
            deg = dlo + rng.below(dhi - dlo + 1)
            while True:
                have0 = rng.bernoulli(0.7)
                have1 = rng.bernoulli(0.7)
                if have0 or have1:
                    break
            ents = {kb + r: 0}
            for j, h in ((0, have0), (1, have1)):
                if h:
                    ents[j] = rng.below(V_RANGE)
            n_other = deg - len(ents)
            for j in rng.sample_distinct(list(range(2, kb + mc)), n_other):
                ents[j] = rng.below(V_RANGE)
            rows.append(ents)
        return rows

    ext = ext_rows()
    while True:
        core = core_rows()
        rows = core + ext
        info_deg = np.zeros(kb, dtype=np.int64)
        for ents in rows:
            for j in ents:
                if j < kb:
                    info_deg[j] += 1
        if np.all(info_deg >= 2):
            break

    R, C, V = [], [], []
    for r, ents in enumerate(rows):
        for j in sorted(ents):
            R.append(r)
            C.append(j)
            V.append(ents[j])
    return BaseGraph(name, mb, nb, kb, mc, npc,
                     np.array(R, dtype=np.int16), np.array(C, dtype=np.int16),
                     np.array(V, dtype=np.int16))


def custom_base_graph(name, mb, nb, kb, mc, n_punct_cols, entries) -> BaseGraph:
    """A base graph from an explicit {(row, col): V} map (test codes)."""
    items = sorted(entries.items())
    return BaseGraph(name, mb, nb, kb, mc, n_punct_cols,
                     np.array([k[0] for k, _ in items], dtype=np.int16),
                     np.array([k[1] for k, _ in items], dtype=np.int16),
                     np.array([v for _, v in items], dtype=np.int16))


def tree_base_graph() -> BaseGraph:
    """A 3 x 7 base matrix whose Tanner graph is a tree (any lift is a forest).

    Rows: {0,1,2,3}, {3,4,5}, {5,6}; columns 3 and 5 are the only shared ones,
    so there is no cycle.  Shifts are arbitrary; lifting a tree gives a forest.
    Used to pin the decoder against brute-force max-log ML.  It has no
    dual-diagonal structure; information columns and parity are not defined.
    """
    ent = {(0, 0): 3, (0, 1): 5, (0, 2): 0, (0, 3): 7,
           (1, 3): 2, (1, 4): 9, (1, 5): 4,
           (2, 5): 1, (2, 6): 6}
    return custom_base_graph("tree", 3, 7, 4, 3, 0, ent)
