"""Puncture flushing + max-log soft demapping + rate dematching (oracle).

Test infrastructure only.  The receiver soft-demodulates, then sets the
confidence of every bit carried by a resource element that URLLC punctured
to "NULL", i.e. LLR 0, so the decoder treats it as an erasure (Sec. VI-D "UE",
"Rx Signal Processing").  The paper's demodulator is a toolbox function whose
algorithm it does not state; this build uses max-log:

    lambda_i(y) = (1 / sigma^2) * [ min_{s: b_i(s)=1} |y - s|^2 - min_{s: b_i(s)=0} |y - s|^2 ]

(positive means bit 0 is more likely), evaluated here by brute force over
all 2^Qm constellation points in float64.  The constellation is the NR-style
recursive Gray QAM: bits b0, b2, .. drive I, b1, b3, .. drive Q; per-axis
amplitude A(c0, c1, ..) = (1 - 2 c0)(2^(q-1) - A(c1, ..)), A(c) = 1 - 2c;
unit average energy.

Rate dematching: the Qm bits of resource element r are rate-matched bits
e = i * (E / Qm) + r (i < Qm) with the row-column interleaver, or
e = r * Qm + i without it; bit e is codeword position t0 + ((k0 + e) mod Ncb),
a circular buffer of Ncb = nb * Z - t0 positions read from the start k0 of the
redundancy version (0 for version 0; versions 1-3 follow NR's table, 3GPP
TS 38.212 rate matching: k0 = (17, 33, 56) Z for a 66 Z buffer and
(13, 25, 43) Z for a 50 Z buffer, the sizes of NR's two base graphs; the paper
sends one transmission per TTI and names no version, Sec. VI-A), and the LLRs
of all bits that land on one position are added (LLR combining); positions
never transmitted hold LLR 0.  The decoded length is n_eff * Z with
n_eff = kb + m_eff and m_eff = min(mb, max(mc, ceil((t0 + last) / Z) - kb)),
t0 = n_punct_cols * Z, last = Ncb if k0 + E > Ncb else k0 + E.

INT modes quantise q = clamp(round_half_away(scale * lambda), -sat, sat).
"""
from __future__ import annotations

import itertools

import numpy as np

NORM2 = {2: 2.0, 4: 10.0, 6: 42.0, 8: 170.0}


def _axis_amp(cbits) -> int:
    """Recursive Gray PAM amplitude of per-axis bits (c0, c1, ...)."""
    if len(cbits) == 1:
        return 1 - 2 * cbits[0]
    return (1 - 2 * cbits[0]) * (2 ** (len(cbits) - 1) - _axis_amp(cbits[1:]))


def constellation(Qm: int):
    """(points complex128 (2^Qm,), labels uint8 (2^Qm, Qm)) with b0 the first label bit."""
    labels = np.array(list(itertools.product((0, 1), repeat=Qm)), dtype=np.uint8)
    pts = np.empty(labels.shape[0], dtype=np.complex128)
    for n, lab in enumerate(labels):
        I = _axis_amp([int(b) for b in lab[0::2]])
        Q = _axis_amp([int(b) for b in lab[1::2]])
        pts[n] = (I + 1j * Q) / np.sqrt(NORM2[Qm])
    return pts, labels


def maxlog_llr(y: np.ndarray, Qm: int, inv_sigma2) -> np.ndarray:
    """Brute-force max-log LLRs: y (n,) complex -> (n, Qm) float64."""
    pts, labels = constellation(Qm)
    y = np.asarray(y, dtype=np.complex128)
    d = np.abs(y[:, None] - pts[None, :]) ** 2          # (n, 2^Qm)
    out = np.empty((y.size, Qm), dtype=np.float64)
    for i in range(Qm):
        one = labels[:, i] == 1
        out[:, i] = d[:, one].min(axis=1) - d[:, ~one].min(axis=1)
    return out * np.asarray(inv_sigma2, dtype=np.float64)


K0_UNITS = {66: (0, 17, 33, 56), 50: (0, 13, 25, 43)}  # k0 / Z per redundancy version, by Ncb / Z


def start_k0(nb, n_punct_cols, Z, rv):
    """Start of redundancy version rv in the circular buffer."""
    if rv == 0:
        return 0
    units = K0_UNITS.get(nb - n_punct_cols)
    if units is None:
        raise ValueError("redundancy versions 1-3 need a 66 Z or 50 Z buffer")
    return units[rv] * Z


def geometry(mb, nb, kb, mc, n_punct_cols, Z, E, rv=0):
    """(t0, m_eff, n_eff) for a code block that transmits E bits of redundancy version rv."""
    t0 = n_punct_cols * Z
    ncb = nb * Z - t0
    k0 = start_k0(nb, n_punct_cols, Z, rv)
    last = ncb if k0 + E > ncb else k0 + E
    cols = -(-(t0 + last) // Z)
    m_eff = min(mb, max(mc, cols - kb))
    return t0, m_eff, kb + m_eff


def bg_geometry(bg, Z, E, rv=0):
    return geometry(bg.mb, bg.nb, bg.kb, bg.mc, bg.n_punct_cols, Z, E, rv)


def rv_of(c) -> int:
    """Redundancy version of a code-block descriptor (bits 1-2 of its flags)."""
    return (int(c["flags"]) >> 1) & 3


def unpack_mask(words: np.ndarray, n: int) -> np.ndarray:
    w = np.asarray(words, dtype=np.uint32)
    bits = (w[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1
    return bits.reshape(-1)[:n].astype(bool)


def demap_cb(y, mask_bits, bg, Z, Qm, E, inv_sigma2, interleave=True, rv=0) -> np.ndarray:
    """One code block: symbols + puncture mask -> LLRs at codeword positions (n_eff*Z,)."""
    t0, m_eff, n_eff = bg_geometry(bg, Z, E, rv)
    k0 = start_k0(bg.nb, bg.n_punct_cols, Z, rv)
    n_re = E // Qm
    lam = maxlog_llr(y[:n_re], Qm, inv_sigma2)          # (n_re, Qm)
    lam[np.asarray(mask_bits[:n_re], dtype=bool)] = 0.0  # puncture flushing
    out = np.zeros(n_eff * Z, dtype=np.float64)
    ncb = bg.nb * Z - t0
    r = np.arange(n_re)
    for i in range(Qm):
        e = i * n_re + r if interleave else r * Qm + i
        np.add.at(out, t0 + (k0 + e) % ncb, lam[:, i])
    return out


def round_half_away(x: np.ndarray) -> np.ndarray:
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def quantise(llr: np.ndarray, scale: float, sat: int) -> np.ndarray:
    return np.clip(round_half_away(np.asarray(llr, dtype=np.float64) * scale), -sat, sat).astype(np.int64)


def demap_workload(w, cb_index=None, interleave=True):
    """LLR buffer (float64, length w.llr_len) for all (or the listed) code blocks."""
    out = np.zeros(w.llr_len, dtype=np.float64)
    idx = range(w.n_cb) if cb_index is None else cb_index
    for i in idx:
        c = w.cbs[i]
        bg = w.bgs[int(c["bg"])]
        Z, Qm, E = int(c["Z"]), int(c["Qm"]), int(c["E"])
        n_re = E // Qm
        ro, mo, lo = int(c["re_offset"]), int(c["mask_word_offset"]), int(c["llr_offset"])
        mbits = unpack_mask(w.mask[mo:mo + -(-n_re // 32)], n_re)
        v = demap_cb(w.sym[ro:ro + n_re], mbits, bg, Z, Qm, E,
                     float(np.float32(c["inv_sigma2"])), interleave, rv_of(c))
        out[lo:lo + v.size] = v
    return out
