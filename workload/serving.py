"""Request streams for the decode service (input generation only).

Config 5's served workload: 40 eMBB users, each sending TB decode requests as
a Poisson process at (by default) one TB per 125 us slot; TBs of U{1..16}
code blocks of the mixed workload's shapes; URLLC puncturing per slot drawn
from a 128-entry codebook.  Codebook entry id = a 7-bit mini-slot mask (bit m:
mini-slot m preempted) with a seeded PRB run of 4-12 PRBs per active
mini-slot; the per-slot id has i.i.d. mini-slot bits of probability
q = 1 - (1 - 0.08)^12 (12 URLLC users with Bernoulli(0.08) arrivals per
mini-slot, the paper's case study).

Requests reference a pool of pre-generated TBs (the transmit chain is too slow
to run per request), laid out in one byte buffer: every symbol first, then
every mask word.
"""
from __future__ import annotations

import numpy as np

from .configs import N_MINISLOT, N_SYM, TBSpec, build, cb_rv, default_bgs, draw_tb_shape, es_n0_sigma2, \
    operating_point_db
from .rng import np_stream

SLOT_NS = 125_000
Q_MINISLOT = 1.0 - (1.0 - 0.08) ** 12


def codebook(n_prb: int, seed: int = 5, size: int = 128):
    """size entries: (7-bit mini-slot mask, [(mini-slot, first PRB, n PRBs)...]) for an n_prb-wide band."""
    rng = np_stream(seed, 11, n_prb)
    book = []
    for cid in range(size):
        runs = []
        for m in range(N_MINISLOT):
            if (cid >> m) & 1:
                ln = min(4 + int(rng.integers(0, 9)), n_prb)
                st = int(rng.integers(0, n_prb - ln + 1))
                runs.append((m, st, ln))
        book.append((cid & 0x7F, runs))
    return book


def draw_pattern_id(rng) -> int:
    bits = rng.random(N_MINISLOT) < Q_MINISLOT
    return int(sum(1 << m for m in range(N_MINISLOT) if bits[m]))


def tb_pool(n_tb: int, seed: int = 5, max_cb: int = 16, snr_range_db=(0.0, 3.0), noiseless: bool = False,
            cb_crc: bool = False, zs=None):
    """A Workload of n_tb independent TBs (one per 'slot'), codebook-punctured; ``cb_crc``: multi-block TBs
    carry a CRC per code block; ``zs``: the lifting sizes drawn from (default: the mixed workload's).

    Es/N0 per TB ~ U[op + snr_range_db[0], op + snr_range_db[1]] with op the
    shape's operating point: the served stream is link-adapted to sit at or
    above the waterfall (the configuration states no SNR).
    """
    bgs = default_bgs()
    rng = np_stream(seed, 3)
    specs, widths, punct, snrs = [], [], [], []
    for t in range(n_tb):
        b, Z, R, Qm, E = draw_tb_shape(rng, bgs) if zs is None else draw_tb_shape(rng, bgs, zs)
        n_cb = 1 + int(rng.integers(0, max_cb))
        n_prb = -(-n_cb * (E // Qm) // (12 * N_SYM))
        snr = operating_point_db(R, Qm) + float(rng.uniform(*snr_range_db))
        specs.append(TBSpec(t, b, Z, Qm, E, n_cb, float(es_n0_sigma2(snr)), 0, 12 * n_prb))
        P = np.zeros((N_SYM, 12 * n_prb), dtype=bool)
        cid = draw_pattern_id(rng)
        for m, st, ln in codebook(n_prb, seed)[cid][1]:
            P[2 * m:2 * m + 2, 12 * st:12 * (st + ln)] = True
        punct.append(P)
        widths.append(12 * n_prb)
        snrs.append(snr)
    w = build("serve_pool", bgs, specs, widths, punct, seed, snr_db=snrs,
              z_set=[32, 64, 128, 256, 384], noiseless=noiseless, cb_crc=cb_crc)
    w.meta.update(dict(max_iter=10, early_term=1, mode="i8"))
    return w


def pool_bytes(w) -> tuple:
    """(pool uint8 array, byte offset of the mask words) for a TB pool workload."""
    sym = np.ascontiguousarray(w.sym, dtype=np.complex64).view(np.uint8)
    mask = np.ascontiguousarray(w.mask, dtype=np.uint32).view(np.uint8)
    pad = (-sym.size) % 16
    return np.concatenate([sym, np.zeros(pad, np.uint8), mask]), sym.size + pad


def tb_records(w, mask_base: int, serve_dtype, pool_index=None, tags=None, result_offsets=None):
    """Request records (serve_dtype fields) for the listed pool TBs."""
    idx = np.arange(w.n_tb) if pool_index is None else np.asarray(pool_index)
    out = np.zeros(idx.size, dtype=serve_dtype)
    for j, t in enumerate(idx):
        tb = w.tbs[t]
        c = w.cbs[int(tb["first_cb"])]
        r = out[j:j + 1]
        for name in ("bg", "Z", "Qm", "E", "inv_sigma2"):
            r[name] = c[name]
        r["n_cb"], r["n_sc"], r["payload_bits"] = tb["n_cb"], tb["n_sc"], tb["payload_bits"]
        r["rv"] = cb_rv(c)
        r["sym_offset"] = int(c["re_offset"]) * 8
        r["mask_offset"] = mask_base + int(c["mask_word_offset"]) * 4
        r["result_offset"] = -1 if result_offsets is None else int(result_offsets[j])
        r["tag"] = j if tags is None else int(tags[j])
    return out


def arrivals(n_slots: int, n_ue: int = 40, tb_per_slot: float = 1.0, n_pool: int = 1, seed: int = 5):
    """(arrival ns, pool TB index) for every request: per UE and slot Poisson(tb_per_slot) requests at the slot start."""
    rng = np_stream(seed, 12)
    counts = rng.poisson(tb_per_slot, size=(n_slots, n_ue))
    per_slot = counts.sum(axis=1)
    t = np.repeat(np.arange(n_slots, dtype=np.int64) * SLOT_NS, per_slot)
    pool_idx = rng.integers(0, n_pool, size=t.size)
    return t, pool_idx
