"""Systematic QC-LDPC encoder and parity check (oracle; test infrastructure only).

The paper encodes with a toolbox LDPC encoder (Sec. VI-A "Tx Signal
Processing") and gives no parameters.  For the seeded dual-diagonal base
matrices of this build the encoder is a closed form: with the core-row
partial sums lambda_r = sum_j P^{s_rj} u_j over the information columns,

    p_0     = sum_r lambda_r
    p_1     = lambda_0 + P^{s_a} p_0            (s_a = raw shift 1, mod Z)
    p_{i+1} = lambda_i + p_i + [i = r_mid] p_0   for i = 1 .. mc-2

and each extension parity block is the sum of its row's other blocks.  Here
(P^s x)[k] = x[(k + s) mod Z].  One codeword at a time, plain loops.
"""
from __future__ import annotations

import numpy as np


def _shift(x: np.ndarray, s: int) -> np.ndarray:
    Z = x.size
    return np.array([x[(k + s) % Z] for k in range(Z)], dtype=np.uint8)


def encode_one(bg, Z: int, info: np.ndarray) -> np.ndarray:
    """info: (kb*Z,) bits -> full codeword (nb*Z,) bits."""
    kb, mc, mb, nb = bg.kb, bg.mc, bg.mb, bg.nb
    blk = [np.zeros(Z, dtype=np.uint8) for _ in range(nb)]
    for j in range(kb):
        blk[j] = np.asarray(info[j * Z:(j + 1) * Z], dtype=np.uint8).copy()
    entries = [(int(r), int(c), int(v)) for r, c, v in zip(bg.row, bg.col, bg.V)]
    lam = [np.zeros(Z, dtype=np.uint8) for _ in range(mc)]
    for r, c, v in entries:
        if r < mc and c < kb:
            lam[r] ^= _shift(blk[c], v % Z)
    p0 = np.zeros(Z, dtype=np.uint8)
    for r in range(mc):
        p0 ^= lam[r]
    blk[kb] = p0
    r_mid = mc // 2
    if mc > 1:
        blk[kb + 1] = lam[0] ^ _shift(p0, 1 % Z)
        for i in range(1, mc - 1):
            blk[kb + i + 1] = lam[i] ^ blk[kb + i] ^ (p0 if i == r_mid else 0)
    for r in range(mc, mb):
        acc = np.zeros(Z, dtype=np.uint8)
        for rr, c, v in entries:
            if rr == r and c != kb + r:
                acc ^= _shift(blk[c], v % Z)
        blk[kb + r] = acc
    return np.concatenate(blk)


def syndrome(bg, Z: int, cw: np.ndarray, rows=None) -> np.ndarray:
    """H c over GF(2) for rows ``rows`` (default all), as an (n_rows*Z,) bit vector.

    Uses only the definition of the lifted matrix: check (r, k) sums the
    variables (c, (k + V_rc mod Z) mod Z) over the row's entries.
    """
    cw = np.asarray(cw, dtype=np.uint8)
    rows = range(bg.mb) if rows is None else rows
    out = []
    for r in rows:
        s = np.zeros(Z, dtype=np.uint8)
        for rr, c, v in zip(bg.row, bg.col, bg.V):
            if rr != r:
                continue
            base = int(c) * Z
            for k in range(Z):
                s[k] ^= cw[base + (k + int(v) % Z) % Z]
        out.append(s)
    return np.concatenate(out) if out else np.zeros(0, dtype=np.uint8)
