"""Request streams for the decode service (input generation only).

The served workload: 40 eMBB users, each sending TB decode requests as a
Poisson process at (by default) one TB per 125 us slot; TBs of U{1..16} code
blocks of the mixed workload's shapes.

URLLC puncturing follows the paper's mini-slot preemption model (Sec. III-A):
a slot has seven mini-slots of two OFDM symbols; a URLLC packet arriving in a
mini-slot preempts subcarriers of whichever eMBB users are scheduled under it
for that mini-slot.  Each slot draws ONE entry of a 128-entry codebook: entry
id = a 7-bit mini-slot mask whose bits are i.i.d. with probability
q = 1 - (1 - 0.08)^12 (12 URLLC users with Bernoulli(0.08) arrivals per
mini-slot, the paper's case study, Sec. VII-B), and per active mini-slot a
seeded run of 4-12 PRBs.  The runs are drawn on a 66-PRB period (the 792
subcarriers of a 120 kHz carrier) and repeat along the slot's grid.  The
slot's TBs sit side by side on that grid, each user a contiguous band of
ceil(RE_tb / 168) PRBs in arrival order, so a burst punctures exactly the
users whose bands lie under it.

The transmit chain is too slow to run per request, so requests reference a
pool of pre-encoded, unpunctured TBs; a request names its slot's codebook
entry and its band's place on the slot's grid, and the service expands the
entry into the punctured resource elements on the device.  ``served_workload``
expands the same requests on the host into an ordinary batch workload (mask
words) for the batch path and the CPU oracle.
"""
from __future__ import annotations

import numpy as np

from .configs import CB_RV_SHIFT, N_MINISLOT, N_SYM, TBSpec, build, default_bgs, draw_tb_shape, es_n0_sigma2, \
    operating_point_db, subset
from .rng import np_stream

SLOT_NS = 125_000
Q_MINISLOT = 1.0 - (1.0 - 0.08) ** 12
CODEBOOK_PRB = 66      # pattern period: one 792-subcarrier carrier
CODEBOOK_SIZE = 128


def codebook(n_prb: int = CODEBOOK_PRB, seed: int = 5, size: int = CODEBOOK_SIZE):
    """size entries: (7-bit mini-slot mask, [(mini-slot, first PRB, n PRBs)...]) on an n_prb-wide period."""
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


def codebook_bitmaps(n_prb: int = CODEBOOK_PRB, seed: int = 5, size: int = CODEBOOK_SIZE) -> np.ndarray:
    """The codebook as the service takes it: uint32 [size][7][ceil(n_prb / 32)], bit p % 32 of word p / 32
    set = PRB p of the period preempted in that mini-slot."""
    wpm = -(-n_prb // 32)
    out = np.zeros((size, N_MINISLOT, wpm), dtype=np.uint32)
    for cid, (_, runs) in enumerate(codebook(n_prb, seed, size)):
        for m, st, ln in runs:
            for p in range(st, st + ln):
                out[cid, m, p >> 5] |= np.uint32(1 << (p & 31))
    return out


def draw_pattern_id(rng) -> int:
    bits = rng.random(N_MINISLOT) < Q_MINISLOT
    return int(sum(1 << m for m in range(N_MINISLOT) if bits[m]))


def tb_pool(n_tb: int, seed: int = 5, max_cb: int = 16, snr_range_db=(0.0, 3.0), noiseless: bool = False,
            cb_crc: bool = False, zs=None, own_band_masks: bool = False):
    """A Workload of n_tb independent TBs (one per 'slot'); ``cb_crc``: multi-block TBs carry a CRC per code
    block; ``zs``: the lifting sizes drawn from (default: the mixed workload's).

    The TBs are unpunctured: requests puncture them through the codebook on
    their slot's grid.  ``own_band_masks``: instead, each TB carries explicit
    mask words of a codebook entry drawn for it alone and laid on its own band
    (inputs for the service's mask-word request form).

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
        if own_band_masks:
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


def tb_records(w, mask_base: int, serve_dtype, pool_index=None, tags=None, result_offsets=None, pattern=None,
               grid_sc=None):
    """Request records (serve_dtype fields) for the listed pool TBs.  ``pattern`` / ``grid_sc`` (per
    record): the codebook entry puncturing the request and its band's first subcarrier on the slot's grid;
    without them a request takes the TB's own mask words (pattern -1)."""
    idx = np.arange(w.n_tb) if pool_index is None else np.asarray(pool_index)
    out = np.zeros(idx.size, dtype=serve_dtype)
    first = w.tbs["first_cb"][idx].astype(np.int64)
    c = w.cbs[first]
    for name in ("bg", "Z", "Qm", "E", "inv_sigma2"):
        out[name] = c[name]
    for name in ("n_cb", "n_sc", "payload_bits"):
        out[name] = w.tbs[name][idx]
    out["rv"] = (c["flags"] >> CB_RV_SHIFT) & 3
    out["sym_offset"] = c["re_offset"].astype(np.int64) * 8
    out["mask_offset"] = mask_base + c["mask_word_offset"].astype(np.int64) * 4
    out["result_offset"] = -1 if result_offsets is None else np.asarray(result_offsets, dtype=np.int64)
    out["tag"] = np.arange(idx.size) if tags is None else np.asarray(tags)
    out["pattern"] = -1 if pattern is None else np.asarray(pattern)
    out["grid_sc"] = 0 if grid_sc is None else np.asarray(grid_sc)
    return out


def arrivals(n_slots: int, n_ue: int = 40, tb_per_slot: float = 1.0, n_pool: int = 1, seed: int = 5):
    """(arrival ns, pool TB index) for every request: per UE and slot Poisson(tb_per_slot) requests at the slot
    start, slot after slot, users in order within a slot."""
    s = slot_stream(n_slots, np.ones(n_pool, np.int64), n_ue, tb_per_slot, seed)
    return s["t_ns"], s["pool"]


def slot_stream(n_slots: int, pool_n_sc, n_ue: int = 40, tb_per_slot: float = 1.0, seed: int = 5) -> dict:
    """The served request stream: per UE and slot Poisson(tb_per_slot) TB requests at the slot start, each
    a uniformly drawn pool TB.  Per slot one codebook entry (i.i.d. mini-slot bits of probability
    Q_MINISLOT); the slot's requests sit side by side on its grid in user order, request i's band starting
    at the sum of the bands (``pool_n_sc``) before it.  Returns arrays over requests: t_ns, pool, pattern,
    grid_sc, slot."""
    pool_n_sc = np.asarray(pool_n_sc, dtype=np.int64)
    rng = np_stream(seed, 12)
    counts = rng.poisson(tb_per_slot, size=(n_slots, n_ue))
    per_slot = counts.sum(axis=1)
    slot = np.repeat(np.arange(n_slots, dtype=np.int64), per_slot)
    t = slot * SLOT_NS
    pool = rng.integers(0, pool_n_sc.size, size=t.size)
    bits = rng.random((n_slots, N_MINISLOT)) < Q_MINISLOT
    pat_slot = (bits.astype(np.int64) << np.arange(N_MINISLOT)).sum(axis=1)
    width = pool_n_sc[pool]
    end = np.cumsum(width)
    start_of_slot = np.concatenate([[0], np.cumsum(per_slot)])[:-1]
    base = np.repeat(end[start_of_slot] - width[start_of_slot], per_slot) if t.size else np.zeros(0, np.int64)
    grid = end - width - base
    return {"t_ns": t, "pool": pool, "pattern": pat_slot[slot], "grid_sc": grid, "slot": slot}


def expand_mask(w, t: int, pattern: int, grid_sc: int, bitmaps: np.ndarray, n_prb: int = CODEBOOK_PRB):
    """Mask words of pool TB t's code blocks (concatenated) under codebook entry ``pattern`` with its band
    starting at subcarrier ``grid_sc`` of the slot's grid: TB resource element i sits on symbol i // n_sc,
    subcarrier grid_sc + i % n_sc, PRB (subcarrier // 12) mod n_prb of the pattern."""
    tb = w.tbs[t]
    first, n_cb, n_sc = int(tb["first_cb"]), int(tb["n_cb"]), int(tb["n_sc"])
    c = w.cbs[first]
    n_re = int(c["E"]) // int(c["Qm"])
    out = []
    for j in range(n_cb):
        i = j * n_re + np.arange(n_re)
        sym = i // n_sc
        if sym.size and sym.max() >= N_SYM:
            raise ValueError("TB does not fit its band in one slot")
        prb = ((grid_sc + i % n_sc) // 12) % n_prb
        hit = (bitmaps[pattern, sym // 2, prb >> 5] >> (prb & 31).astype(np.uint32)) & 1
        bits = np.zeros(-(-n_re // 32) * 32, dtype=np.uint32)
        bits[:n_re] = hit
        out.append((bits.reshape(-1, 32) << np.arange(32, dtype=np.uint32)).sum(axis=1, dtype=np.uint64)
                   .astype(np.uint32))
    return out


def served_workload(w, pool_index, pattern, grid_sc, bitmaps: np.ndarray, n_prb: int = CODEBOOK_PRB):
    """The listed requests as an ordinary workload (one TB per request, in order), their puncturing
    expanded on the host into mask words: the inputs the batch path and the CPU oracle decode."""
    sub = subset(w, list(pool_index))
    words = []
    for t, p, g in zip(pool_index, pattern, grid_sc):
        words.extend(expand_mask(w, int(t), int(p), int(g), bitmaps, n_prb))
    sub.mask = np.concatenate(words) if words else np.zeros(0, np.uint32)
    assert sub.mask.size == sum(x.size for x in words)
    return sub
