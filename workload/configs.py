"""Synthetic slots shaped like the paper's workloads (input generation only).

The paper's system model (Sec. III-A) divides a TTI into one slot of seven
mini-slots of two OFDM symbols; eMBB user ``e`` holds ``n_e`` subcarriers for
the slot; URLLC packets of ``L`` subcarriers preempt eMBB resource elements
in a mini-slot; the puncturing vector ``y(t, tau)`` counts how many of each
user's subcarriers are taken.  The receiver is told which resource elements
were punctured (Sec. VI-A, "SC Puncturing Mapping").

A ``Workload`` holds everything one batch of the receive path consumes, laid
out exactly as the C-ABI wants it:

* ``cbs`` / ``tbs``: descriptor arrays (dtypes ``CB_DTYPE`` / ``TB_DTYPE``
  match ``ldpc_cb_desc`` / ``ldpc_tb_desc``);
* ``sym``: received complex64 symbols of every code block, concatenated;
* ``mask``: one bit per resource element (bit ``r % 32`` of word ``r // 32``
  of the block's mask words), 1 = punctured by URLLC;
* ``slot_N``: subcarriers of each slot (the ``N`` of the reward);
* ``info_words``: the transmitted information bits of every code block, packed
  like the decoder's output (bit ``i`` of a block is bit ``i % 32`` of word
  ``i // 32``).

Resource-element mapping: each TB owns a band of ``w`` subcarriers for the
whole slot; its resource elements are filled frequency-first then symbol by
symbol, code block after code block; mini-slot ``m`` is symbols ``2m, 2m+1``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import tx
from .basegraph import BaseGraph, make_base_graph
from .rng import np_stream

N_SYM = 14
N_MINISLOT = 7

CB_DTYPE = np.dtype([
    ("bg", "<i4"), ("Z", "<i4"), ("Qm", "<i4"), ("E", "<i4"),
    ("re_offset", "<i8"), ("mask_word_offset", "<i8"),
    ("llr_offset", "<i8"), ("bits_word_offset", "<i8"),
    ("inv_sigma2", "<f4"), ("flags", "<i4"),
])
CB_FLAG_CRC24B = 1  # the code block's last 24 bits are a CRC (0x800063) of its first K - 24
CB_RV_SHIFT = 1     # flags bits 1-2: the redundancy version sent
assert CB_DTYPE.itemsize == 56

TB_DTYPE = np.dtype([
    ("first_cb", "<i4"), ("n_cb", "<i4"), ("n_sc", "<i4"), ("slot", "<i4"),
    ("payload_bits", "<i4"),
])
assert TB_DTYPE.itemsize == 20

BG_NAMES = ("bg1", "bg2", "tiny")


@dataclass
class TBSpec:
    slot: int
    bg: int            # index into Workload.bgs
    Z: int
    Qm: int
    E: int
    n_cb: int
    sigma2: float
    sc0: int           # first subcarrier of the band in the slot grid
    width: int         # band width in subcarriers (= n_e, the SCs of the allocation)
    rv: int = 0        # redundancy version of every code block of the TB


@dataclass
class Workload:
    name: str
    bgs: list
    z_set: list
    cbs: np.ndarray
    tbs: np.ndarray
    slot_N: np.ndarray
    sym: np.ndarray
    mask: np.ndarray
    info_words: np.ndarray
    llr_len: int
    bits_words: int
    snr_db: np.ndarray = field(default=None)      # per CB, for BLER bookkeeping
    meta: dict = field(default_factory=dict)

    @property
    def n_cb(self) -> int:
        return int(self.cbs.size)

    @property
    def n_tb(self) -> int:
        return int(self.tbs.size)

    @property
    def n_slots(self) -> int:
        return int(self.slot_N.size)

    def info_bits_total(self) -> int:
        return int(sum(self.bgs[c["bg"]].kb * int(c["Z"]) for c in self.cbs))

    def cb_geometry(self, i: int):
        """(BaseGraph, Z, t0, m_eff, n_eff) of code block i."""
        c = self.cbs[i]
        bg = self.bgs[int(c["bg"])]
        Z, E, rv = int(c["Z"]), int(c["E"]), cb_rv(c)
        return bg, Z, bg.t0(Z), bg.m_eff(Z, E, rv), bg.n_eff(Z, E, rv)


def cb_rv(c) -> int:
    """Redundancy version of a code-block descriptor."""
    return (int(c["flags"]) >> CB_RV_SHIFT) & 3


def default_bgs() -> list:
    return [make_base_graph(n) for n in BG_NAMES]


def es_n0_sigma2(snr_db):
    """Es/N0 in dB -> noise variance per unit-energy symbol."""
    return 10.0 ** (-np.asarray(snr_db, dtype=np.float64) / 10.0)


def eb_n0_sigma2(ebn0_db, R, Qm):
    return 1.0 / (R * Qm * 10.0 ** (np.asarray(ebn0_db, dtype=np.float64) / 10.0))


def _pack_bits(bits: np.ndarray) -> np.ndarray:
    """(n, 32m) uint8 bits -> (n, m) uint32, bit i -> bit i % 32 of word i // 32."""
    n, L = bits.shape
    b = bits.reshape(n, L // 32, 32).astype(np.uint32)
    return (b << np.arange(32, dtype=np.uint32)).sum(axis=2, dtype=np.uint64).astype(np.uint32)


def build(name: str, bgs: list, specs: list, slot_widths: list, punct: list, seed: int,
          interleave: bool = True, snr_db=None, z_set=None, noiseless: bool = False,
          cb_crc: bool = False) -> Workload:
    """Run the Tx chain for ``specs`` and lay the result out for the receiver.

    ``punct[s]`` is a (14, slot_widths[s]) boolean map of slot ``s``'s punctured
    resource elements.  ``noiseless`` skips the AWGN (tests).  ``cb_crc``: every
    TB of more than one code block carries a CRC-24 (0x800063) per code block,
    so its payload is A = n_cb (K - 24) - 24 bits; single-block TBs have none.
    """
    n_tb = len(specs)
    rng_payload = np_stream(seed, 1)
    rng_noise = np_stream(seed, 2)

    # ---- descriptors and offsets
    cb_rows, tb_rows, per_cb = [], [], []
    re_off = mask_off = llr_off = bits_off = 0
    for t, sp in enumerate(specs):
        bg = bgs[sp.bg]
        K = bg.kb * sp.Z
        if K % 32:
            raise ValueError("K must be a multiple of 32")
        if sp.E % sp.Qm:
            raise ValueError("E must be a multiple of Qm")
        n_re = sp.E // sp.Qm
        n_eff = bg.n_eff(sp.Z, sp.E, sp.rv)
        seg = cb_crc and sp.n_cb > 1
        tb_rows.append((len(cb_rows), sp.n_cb, sp.width, sp.slot, sp.n_cb * (K - 24 * seg) - 24))
        for j in range(sp.n_cb):
            cb_rows.append((sp.bg, sp.Z, sp.Qm, sp.E, re_off, mask_off, llr_off, bits_off,
                            np.float32(1.0 / sp.sigma2), (CB_FLAG_CRC24B if seg else 0) | (sp.rv << CB_RV_SHIFT)))
            per_cb.append((t, j, n_re))
            re_off += n_re
            mask_off += -(-n_re // 32)
            llr_off += n_eff * sp.Z
            bits_off += K // 32
    cbs = np.array(cb_rows, dtype=CB_DTYPE)
    tbs = np.array(tb_rows, dtype=TB_DTYPE)

    sym = np.zeros(re_off, dtype=np.complex64)
    mask = np.zeros(mask_off, dtype=np.uint32)
    info_words = np.zeros(bits_off, dtype=np.uint32)

    # ---- payload + CRC per TB, split into code blocks
    cb_info = [None] * len(cb_rows)
    by_A: dict[int, list] = {}
    for t, sp in enumerate(specs):
        by_A.setdefault(int(tbs[t]["payload_bits"]), []).append(t)
    for A, ts in sorted(by_A.items()):
        payload = rng_payload.integers(0, 2, size=(len(ts), A), dtype=np.uint8)
        tbbits = tx.crc24_attach(payload)
        for row, t in enumerate(ts):
            sp = specs[t]
            K = bgs[sp.bg].kb * sp.Z
            first = int(tbs[t]["first_cb"])
            if cbs[first]["flags"] & CB_FLAG_CRC24B:
                segs = tbbits[row].reshape(sp.n_cb, K - 24)
                cw_info = tx.crc24_attach(segs, tx.CRC24B_POLY)
                for j in range(sp.n_cb):
                    cb_info[first + j] = cw_info[j]
            else:
                for j in range(sp.n_cb):
                    cb_info[first + j] = tbbits[row, j * K:(j + 1) * K]

    # ---- encode / rate match / modulate per shape group
    groups: dict[tuple, list] = {}
    for i, c in enumerate(cbs):
        groups.setdefault((int(c["bg"]), int(c["Z"]), int(c["E"]), int(c["Qm"]), cb_rv(c)), []).append(i)
    for (b, Z, E, Qm, rv), idx in sorted(groups.items()):
        bg = bgs[b]
        info = np.stack([cb_info[i] for i in idx])
        k0 = bg.k0(Z, rv)
        # columns up to the last position sent (a transmission that wraps the buffer reaches them all)
        n_cols = bg.nb if k0 + E > bg.ncb(Z) else -(-(bg.t0(Z) + k0 + E) // Z)
        cw = tx.encode(bg, Z, info, n_cols=n_cols)
        e = tx.rate_match(bg, Z, cw, E, rv)
        re_bits = tx.interleave(e, Qm, interleave)
        x = tx.qam_map(re_bits)  # (B, n_re)
        sig2 = np.array([1.0 / float(cbs[i]["inv_sigma2"]) for i in idx])
        y = x if noiseless else tx.awgn(x, sig2[:, None], rng_noise)
        info_w = _pack_bits(info)
        for row, i in enumerate(idx):
            o = int(cbs[i]["re_offset"])
            sym[o:o + y.shape[1]] = y[row]
            w = int(cbs[i]["bits_word_offset"])
            info_words[w:w + info_w.shape[1]] = info_w[row]

    # ---- resource-element mapping and puncturing
    us = tx.urllc_symbol()
    for i, (t, j, n_re) in enumerate(per_cb):
        sp = specs[t]
        tr = j * n_re + np.arange(n_re)               # TB-level RE index
        symb = tr // sp.width
        sc = sp.sc0 + tr % sp.width
        if symb.size and symb.max() >= N_SYM:
            raise ValueError("TB does not fit its band in one slot")
        hit = punct[sp.slot][symb, sc]
        o = int(cbs[i]["re_offset"])
        sym[o:o + n_re][hit] = us
        words = np.zeros(-(-n_re // 32) * 32, dtype=np.uint8)
        words[:n_re] = hit
        mw = int(cbs[i]["mask_word_offset"])
        mask[mw:mw + words.size // 32] = _pack_bits(words[None, :])[0]

    snr = None if snr_db is None else np.repeat(np.asarray(snr_db, dtype=np.float64),
                                               [s.n_cb for s in specs])
    zs = sorted({int(c["Z"]) for c in cbs}) if z_set is None else list(z_set)
    return Workload(name, bgs, zs, cbs, tbs, np.array([w for w in slot_widths], dtype=np.int32),
                    sym, mask, info_words, llr_off, bits_off, snr_db=snr)


# ============================================================================ configs
def tiny_fp32(n_per_point: int = 1000, ebn0_points=(0, 1, 2, 3, 4), seed: int = 0,
              p_minislot: float = 0.2, frac: float = 0.25, noiseless: bool = False) -> Workload:
    """8x16 base matrix, Z=16, rate 1/2 with all N=256 bits sent, QPSK, Eb/N0 points.

    One codeword per slot on a 10-SC x 14-symbol grid (128 of 140 REs used).
    Each mini-slot is hit with probability ``p_minislot``; a hit punctures
    round(frac * n) of the codeword's n resource elements in that mini-slot,
    chosen uniformly.
    """
    bgs = default_bgs()
    Z, Qm, E = 16, 2, 256
    width = 10
    rng = np_stream(seed, 3)
    specs, widths, punct, snrs = [], [], [], []
    for p_i, eb in enumerate(ebn0_points):
        s2 = float(eb_n0_sigma2(eb, 0.5, Qm))
        for _ in range(n_per_point):
            slot = len(specs)
            specs.append(TBSpec(slot, 2, Z, Qm, E, 1, s2, 0, width))
            P = np.zeros((N_SYM, width), dtype=bool)
            used = np.zeros((N_SYM, width), dtype=bool)
            used.reshape(-1)[:E // Qm] = True
            for m in range(N_MINISLOT):
                if rng.random() < p_minislot:
                    cells = np.flatnonzero(used[2 * m:2 * m + 2].reshape(-1))
                    k = int(np.floor(frac * cells.size + 0.5))
                    pick = rng.choice(cells, size=k, replace=False)
                    sub = P[2 * m:2 * m + 2].reshape(-1)
                    sub[pick] = True
                    P[2 * m:2 * m + 2] = sub.reshape(2, width)
            punct.append(P)
            widths.append(width)
            snrs.append(eb)
    w = build("tiny_fp32", bgs, specs, widths, punct, seed, snr_db=snrs, noiseless=noiseless)
    w.meta.update(dict(name="tiny", max_iter=8, early_term=0, mode="f32", offset=0.5))
    return w


CFG2_PRB = 66
CFG2_UE_PRB = 26


def large_fp32(n_cw: int = 4096, snr_points=(6, 7, 8, 9, 10, 11, 12), seed: int = 2,
               with_urllc: bool = True, noiseless: bool = False) -> Workload:
    """BG1-shaped 46x68, Z=384, K=8448, rate 1/2 (E=16896), 16-QAM.

    Slots of 66 PRBs x 14 symbols; two users per slot with 26-PRB bands
    (PRBs [0,26) and [26,52)), one code block each.  Codeword ``i`` gets
    Es/N0 ``snr_points[i % len]``.  Per slot, 1-3 distinct mini-slots are
    preempted, each by one contiguous run of 4-12 PRBs at a uniform start.
    """
    bgs = default_bgs()
    Z, Qm = 384, 4
    K = bgs[0].kb * Z
    E = Qm * int(round(K / (0.5 * Qm)))
    rng = np_stream(seed, 3)
    n_slots = -(-n_cw // 2)
    width_slot = CFG2_PRB * 12
    specs, punct, snrs = [], [], []
    for s in range(n_slots):
        P = np.zeros((N_SYM, width_slot), dtype=bool)
        if with_urllc:
            n_ms = 1 + int(rng.integers(0, 3))
            for m in rng.choice(N_MINISLOT, size=n_ms, replace=False):
                ln = 4 + int(rng.integers(0, 9))
                st = int(rng.integers(0, CFG2_PRB - ln + 1))
                P[2 * m:2 * m + 2, 12 * st:12 * (st + ln)] = True
        punct.append(P)
        for u in range(2):
            i = 2 * s + u
            if i >= n_cw:
                break
            snr = snr_points[i % len(snr_points)]
            specs.append(TBSpec(s, 0, Z, Qm, E, 1, float(es_n0_sigma2(snr)),
                                12 * CFG2_UE_PRB * u, 12 * CFG2_UE_PRB))
            snrs.append(snr)
    w = build("large_fp32", bgs, specs, [width_slot] * n_slots, punct, seed, snr_db=snrs,
              noiseless=noiseless)
    w.meta.update(dict(name="large", max_iter=10, early_term=1, mode="f32", offset=0.5))
    return w


MIX_Z = (32, 64, 128, 256, 384)
MIX_QM = (2, 4, 6, 8)


def operating_point_db(R: float, Qm: int) -> float:
    """Es/N0 near a code's waterfall: Shannon's bound for R*Qm bit/symbol plus 3 dB.

    3 dB is the measured gap of these codes at ~10 % code-block error rate
    (BG1-shaped, R = 1/2, 16-QAM, URLLC masks: 10 % BLER at 8.0 dB against a
    4.8 dB bound; see results/precision_sweep_large.md).
    """
    return float(10.0 * np.log10(2.0 ** (R * Qm) - 1.0) + 3.0)


_PEELS: dict = {}


def _peels(bg, Z: int, E: int) -> bool:
    key = (bg.sha256(), Z, E)
    if key not in _PEELS:
        _PEELS[key] = bg.peels_to_information(Z, E)
    return _PEELS[key]


def draw_tb_shape(rng, bgs, zs=MIX_Z):
    """One TB's (bg, Z, R, Qm, E) for the mixed workload (Z from ``zs``).  Rates below kb/(nb-2)
    (BG1-shaped: 1/3) send more bits than the circular buffer holds, so their rate matching wraps it
    (repetition).  R is redrawn while the rate-matched code cannot recover its information bits even
    without noise (``BaseGraph.peels_to_information``: at the highest rates every decoded row of the
    seeded graphs holds both punctured columns -- BG1-shaped R >= 0.88, BG2-shaped R >= 0.83)."""
    b = int(rng.integers(0, 2))
    bg = bgs[b]
    Z = int(zs[int(rng.integers(0, len(zs)))])
    Qm = int(MIX_QM[int(rng.integers(0, len(MIX_QM)))])
    K = bg.kb * Z
    while True:
        R = float(rng.uniform(0.3, 0.9))
        E = Qm * int(round(K / (R * Qm)))
        if _peels(bg, Z, E):
            return b, Z, R, Qm, E


def mixed(n_slots: int = 512, ues_per_slot: int = 8, max_cb: int = 8, seed: int = 3,
          spread_db: float = 3.0, noiseless: bool = False, cb_crc: bool = False) -> Workload:
    """Uneven batch: per TB, BG in {bg1, bg2}, Z in {32..384}, R ~ U[0.3, 0.9] (BG1-shaped below 1/3
    repeats the circular buffer), Qm in {2,4,6,8}.

    Each UE has one TB of U{1..max_cb} code blocks per slot, with a contiguous
    PRB band of ceil(RE_tb / 168) PRBs; the slot grid is the concatenation of
    the bands.  Es/N0 per TB ~ U[op - spread, op + spread] around
    ``operating_point_db``.  Each slot carries 1-4 URLLC arrivals (Poisson(2)
    redrawn until in [1, 4]), each on a uniform mini-slot and 4-12 contiguous
    PRBs at a uniform start.  ``cb_crc``: TBs of more than one code block carry
    a CRC per code block (payload n_cb (K - 24) - 24 bits).
    """
    bgs = default_bgs()
    rng = np_stream(seed, 3)
    specs, widths, punct, snrs = [], [], [], []
    for s in range(n_slots):
        sc0 = 0
        slot_specs = []
        for u in range(ues_per_slot):
            b, Z, R, Qm, E = draw_tb_shape(rng, bgs)
            n_cb = 1 + int(rng.integers(0, max_cb))
            re_tb = n_cb * (E // Qm)
            n_prb = -(-re_tb // (12 * N_SYM))
            snr = operating_point_db(R, Qm) + float(rng.uniform(-spread_db, spread_db))
            slot_specs.append(TBSpec(s, b, Z, Qm, E, n_cb, float(es_n0_sigma2(snr)), sc0, 12 * n_prb))
            snrs.append(snr)
            sc0 += 12 * n_prb
        n_prb_slot = sc0 // 12
        P = np.zeros((N_SYM, sc0), dtype=bool)
        while True:
            k = int(rng.poisson(2.0))
            if 1 <= k <= 4:
                break
        for _ in range(k):
            m = int(rng.integers(0, N_MINISLOT))
            ln = min(4 + int(rng.integers(0, 9)), n_prb_slot)
            st = int(rng.integers(0, n_prb_slot - ln + 1))
            P[2 * m:2 * m + 2, 12 * st:12 * (st + ln)] = True
        specs.extend(slot_specs)
        widths.append(sc0)
        punct.append(P)
    w = build("mixed", bgs, specs, widths, punct, seed, snr_db=snrs, z_set=list(MIX_Z),
              noiseless=noiseless, cb_crc=cb_crc)
    w.meta.update(dict(name="mixed", max_iter=10, early_term=1, mode="i8", offset=0.5))
    return w


def repetition(n_per_shape: int = 24, seed: int = 12, noiseless: bool = False) -> Workload:
    """Code blocks whose rate matching wraps the circular buffer (E > Ncb = nb*Z - t0): BG1-shaped Z=64 at
    R = 0.3 and BG2-shaped Z=32 at R = 0.15, 16-QAM, one code block per TB and slot, Es/N0 around the
    operating point, 1-2 URLLC mini-slot runs per slot."""
    bgs = default_bgs()
    rng = np_stream(seed, 4)
    specs, widths, punct, snrs = [], [], [], []
    for b, Z, R in [(0, 64, 0.3), (1, 32, 0.15)]:
        bg = bgs[b]
        Qm = 4
        K = bg.kb * Z
        E = Qm * int(round(K / (R * Qm)))
        assert bg.nb * Z - bg.t0(Z) < E <= 2 * (bg.nb * Z - bg.t0(Z))
        n_re = E // Qm
        width = 12 * -(-n_re // (12 * N_SYM))
        for _ in range(n_per_shape):
            slot = len(specs)
            snr = operating_point_db(R, Qm) + float(rng.uniform(-1.0, 2.0))
            specs.append(TBSpec(slot, b, Z, Qm, E, 1, float(es_n0_sigma2(snr)), 0, width))
            snrs.append(snr)
            P = np.zeros((N_SYM, width), dtype=bool)
            for _ in range(1 + int(rng.integers(0, 2))):
                m = int(rng.integers(0, N_MINISLOT))
                ln = min(12 * (1 + int(rng.integers(0, 3))), width)
                st = int(rng.integers(0, width - ln + 1))
                P[2 * m:2 * m + 2, st:st + ln] = True
            punct.append(P)
            widths.append(width)
    w = build("repetition", bgs, specs, widths, punct, seed, snr_db=snrs, noiseless=noiseless)
    w.meta.update(dict(name="repetition", max_iter=10, early_term=1, mode="f32", offset=0.5))
    return w


def segmented(n_tb: int = 24, seed: int = 13, spread_db=(-1.0, 2.0), noiseless: bool = False) -> Workload:
    """Segmented TBs with a CRC per code block: 2-4 code blocks each, BG1-shaped Z=32 or BG2-shaped
    Z in {32, 64}, R ~ U[0.4, 0.6], QPSK or 16-QAM, Es/N0 around the operating point; one TB per slot,
    1-2 URLLC mini-slot runs of 1-3 PRBs per slot."""
    bgs = default_bgs()
    rng = np_stream(seed, 5)
    specs, widths, punct, snrs = [], [], [], []
    shapes = [(0, 32), (1, 32), (1, 64)]
    for t in range(n_tb):
        b, Z = shapes[int(rng.integers(0, len(shapes)))]
        Qm = (2, 4)[int(rng.integers(0, 2))]
        R = float(rng.uniform(0.4, 0.6))
        K = bgs[b].kb * Z
        E = Qm * int(round(K / (R * Qm)))
        n_cb = 2 + int(rng.integers(0, 3))
        width = 12 * -(-n_cb * (E // Qm) // (12 * N_SYM))
        snr = operating_point_db(R, Qm) + float(rng.uniform(*spread_db))
        specs.append(TBSpec(t, b, Z, Qm, E, n_cb, float(es_n0_sigma2(snr)), 0, width))
        snrs.append(snr)
        P = np.zeros((N_SYM, width), dtype=bool)
        for _ in range(1 + int(rng.integers(0, 2))):
            m = int(rng.integers(0, N_MINISLOT))
            ln = min(12 * (1 + int(rng.integers(0, 3))), width)
            st = int(rng.integers(0, width - ln + 1))
            P[2 * m:2 * m + 2, st:st + ln] = True
        punct.append(P)
        widths.append(width)
    w = build("segmented", bgs, specs, widths, punct, seed, snr_db=snrs, noiseless=noiseless, cb_crc=True)
    w.meta.update(dict(name="segmented", max_iter=10, early_term=1, mode="f32", offset=0.5))
    return w


def redundancy_versions(n_per: int = 3, seed: int = 14, noiseless: bool = False, rates=(0.5, 0.3)) -> Workload:
    """Code blocks of every redundancy version: BG1-shaped Z=64 and BG2-shaped Z=32, R in ``rates``,
    16-QAM, one code block per TB and slot, Es/N0 0-3 dB above the operating point, one URLLC mini-slot
    run per slot.  Versions 1-3 start inside the circular buffer (leaving systematic columns unsent) and
    wrap it."""
    bgs = default_bgs()
    rng = np_stream(seed, 6)
    specs, widths, punct, snrs = [], [], [], []
    for b, Z in [(0, 64), (1, 32)]:
        bg = bgs[b]
        for R in rates:
            Qm = 4
            K = bg.kb * Z
            E = Qm * int(round(K / (R * Qm)))
            n_re = E // Qm
            width = 12 * -(-n_re // (12 * N_SYM))
            for rv in range(4):
                for _ in range(n_per):
                    slot = len(specs)
                    snr = operating_point_db(R, Qm) + float(rng.uniform(0.0, 3.0))
                    specs.append(TBSpec(slot, b, Z, Qm, E, 1, float(es_n0_sigma2(snr)), 0, width, rv))
                    snrs.append(snr)
                    P = np.zeros((N_SYM, width), dtype=bool)
                    m = int(rng.integers(0, N_MINISLOT))
                    ln = min(12, width)
                    st = int(rng.integers(0, width - ln + 1))
                    P[2 * m:2 * m + 2, st:st + ln] = True
                    punct.append(P)
                    widths.append(width)
    w = build("redundancy", bgs, specs, widths, punct, seed, snr_db=snrs, noiseless=noiseless)
    w.meta.update(dict(name="redundancy", max_iter=10, early_term=1, mode="f32", offset=0.5))
    return w


def subset(w: Workload, tb_index) -> Workload:
    """A workload holding only the listed transport blocks (offsets re-based, slots renumbered)."""
    tb_index = list(tb_index)
    cb_rows, tb_rows, slots = [], [], {}
    sym, mask, info = [], [], []
    re_off = mask_off = llr_off = bits_off = 0
    snr = []
    for t in tb_index:
        tb = w.tbs[t]
        s_new = slots.setdefault(int(tb["slot"]), len(slots))
        tb_rows.append((len(cb_rows), int(tb["n_cb"]), int(tb["n_sc"]), s_new, int(tb["payload_bits"])))
        for i in range(int(tb["first_cb"]), int(tb["first_cb"]) + int(tb["n_cb"])):
            c = w.cbs[i]
            bg, Z, t0, m_eff, n_eff = w.cb_geometry(i)
            n_re = int(c["E"]) // int(c["Qm"])
            nmw = -(-n_re // 32)
            kw = bg.kb * Z // 32
            sym.append(w.sym[int(c["re_offset"]):int(c["re_offset"]) + n_re])
            mask.append(w.mask[int(c["mask_word_offset"]):int(c["mask_word_offset"]) + nmw])
            info.append(w.info_words[int(c["bits_word_offset"]):int(c["bits_word_offset"]) + kw])
            cb_rows.append((int(c["bg"]), Z, int(c["Qm"]), int(c["E"]), re_off, mask_off, llr_off, bits_off,
                            c["inv_sigma2"], int(c["flags"])))
            if w.snr_db is not None:
                snr.append(w.snr_db[i])
            re_off += n_re
            mask_off += nmw
            llr_off += n_eff * Z
            bits_off += kw
    slot_N = np.zeros(len(slots), dtype=np.int32)
    for old, new in slots.items():
        slot_N[new] = w.slot_N[old]
    out = Workload(w.name + "_subset", w.bgs, w.z_set, np.array(cb_rows, dtype=CB_DTYPE),
                   np.array(tb_rows, dtype=TB_DTYPE), slot_N,
                   np.concatenate(sym) if sym else np.zeros(0, np.complex64),
                   np.concatenate(mask) if mask else np.zeros(0, np.uint32),
                   np.concatenate(info) if info else np.zeros(0, np.uint32), llr_off, bits_off,
                   snr_db=np.array(snr) if snr else None, meta=dict(w.meta))
    return out
