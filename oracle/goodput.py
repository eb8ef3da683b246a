"""Transport-block CRC check, goodput (eq. 1) and reward (eq. 2) (oracle; test infrastructure only).

d_e = 1 when eMBB user e's packet in the TTI decodes correctly, else 0
(Sec. III-B).  Per slot (TTI) t with users e holding n_e subcarriers out of N:

    goodput_sc(t) = sum_e d_e * n_e                       (Sec. III-B, eq. 1)
    r(t)          = (1 / N) * sum_e (d_e - 1) * n_e       (Sec. V-A, eq. 2)

so r(t) lies in [-1, 0]: 0 when every user decodes, -1 when all fail and the
users fill the N subcarriers.  goodput_bits(t) = sum_e d_e * A_e counts the
delivered payload bits.  A TB's bits are its code blocks' K information bits
in code-block order, less the last 24 of each block that carries its own CRC;
its A payload bits plus 24 CRC bits are checked with ``crc.tb_ok``, and d_e = 1
needs that check and every code-block CRC of the TB (``crc.cb_ok``) to pass:
all CRC bits the transmitter attached must match.
"""
from __future__ import annotations

import numpy as np

from . import crc


def unpack_words(words: np.ndarray, n_bits: int) -> np.ndarray:
    w = np.asarray(words, dtype=np.uint32)
    b = (w[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1
    return b.reshape(-1)[:n_bits].astype(np.uint8)


def cb_bits(w, words, i) -> np.ndarray:
    """The K received information bits of code block ``i``."""
    c = w.cbs[i]
    K = w.bgs[int(c["bg"])].kb * int(c["Z"])
    o = int(c["bits_word_offset"])
    return unpack_words(words[o:o + K // 32], K)


def tb_bitstream(w, words, t) -> np.ndarray:
    """The (A + 24) received bits of TB ``t`` from the packed decoder output."""
    tb = w.tbs[t]
    parts = []
    for i in range(int(tb["first_cb"]), int(tb["first_cb"]) + int(tb["n_cb"])):
        b = cb_bits(w, words, i)
        parts.append(b[:b.size - 24] if int(w.cbs[i]["flags"]) & 1 else b)
    return np.concatenate(parts)


def tb_crc_goodput(w, words, tb_index=None):
    """(d uint8 (n_tb,), goodput_bits int64 (n_slots,), goodput_sc int64 (n_slots,), reward float64 (n_slots,)).

    ``tb_index``: check only the listed TBs; the others get d = 0 and the per-slot sums cover the listed
    ones only."""
    d = np.zeros(w.n_tb, dtype=np.uint8)
    listed = range(w.n_tb) if tb_index is None else [int(t) for t in tb_index]
    by_len: dict = {}
    for t in listed:
        s = tb_bitstream(w, words, t)
        by_len.setdefault(s.size, []).append((t, s))
    for _, items in by_len.items():
        ts = [t for t, _ in items]
        d[ts] = crc.tb_ok(np.stack([s for _, s in items]))
    for t in listed:
        tb = w.tbs[t]
        for i in range(int(tb["first_cb"]), int(tb["first_cb"]) + int(tb["n_cb"])):
            if int(w.cbs[i]["flags"]) & 1 and not crc.cb_ok(cb_bits(w, words, i))[0]:
                d[t] = 0
    n_slots = w.n_slots
    gb = np.zeros(n_slots, dtype=np.int64)
    gs = np.zeros(n_slots, dtype=np.int64)
    fail_sc = np.zeros(n_slots, dtype=np.int64)
    for t in listed:
        tb = w.tbs[t]
        s = int(tb["slot"])
        n_e = int(tb["n_sc"])
        gb[s] += int(d[t]) * int(tb["payload_bits"])
        gs[s] += int(d[t]) * n_e
        fail_sc[s] += (int(d[t]) - 1) * n_e
    reward = fail_sc / np.asarray(w.slot_N, dtype=np.float64)
    return d, gb, gs, reward


def reward_closed_form(d, n, N) -> float:
    """Eq. 2 for one slot, written out: (1/N) * sum_e (d_e - 1) * n_e."""
    return float(sum((int(de) - 1) * int(ne) for de, ne in zip(d, n))) / float(N)


def goodput_closed_form(d, n) -> int:
    """Eq. 1's per-TTI goodput, written out: sum_e d_e * n_e."""
    return int(sum(int(de) * int(ne) for de, ne in zip(d, n)))
