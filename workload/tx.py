"""Transmit chain for the synthetic workloads (input generation only).

The paper's transmitter appends CRC bits to random eMBB data, LDPC-encodes,
rate-matches, punctures the resource elements taken by URLLC, and modulates
(Sec. VI-A, "eMBB Traffic Generator" and "Tx Signal Processing").  This module
produces those transmitted symbols for the tests and the benchmark.  It holds
none of the receiver's arithmetic: no demapping, no decoding, no CRC check.

Conventions fixed here (and restated by the receiver side):

* CRC-24 generator 0x864CFB (degree 24), register starting at 0, message bits
  taken most-significant (first) bit first, no reflection, no final xor; one
  CRC per transport block (TB) of ``A`` payload bits.  The TB's ``A + 24``
  bits fill its code blocks in order, ``K = kb * Z`` bits each, with no filler.
* Per-code-block CRC (optional, TBs of more than one code block): each code
  block takes ``K - 24`` of the TB's bits and appends 24 CRC bits of
  generator 0x800063 over them (same conventions), so ``A + 24 = n_cb (K - 24)``.
* Systematic encoding: ``c[0:K] = info``; core parity by the dual-diagonal
  closed form; extension parity is the sum of its row's other blocks.
* Rate matching: bit ``e`` of the ``E`` transmitted bits is codeword position
  ``t0 + ((k0 + e) mod Ncb)`` with ``t0 = n_punct_cols * Z``, ``Ncb = nb * Z -
  t0`` and ``k0`` the start of the redundancy version (0 for version 0; NR's
  table for versions 1-3, see ``BaseGraph.k0``): positions ``[t0, t0 + E)`` for
  version 0 and ``E <= Ncb``, around the buffer otherwise (``E <= 2 Ncb``).
* Interleaver (flag, default on): the E bits are written row-wise into ``Qm``
  rows of ``E / Qm`` and read column-wise, so resource element ``r`` carries
  bits ``e[i * (E / Qm) + r]`` for ``i < Qm``.
* Gray QAM, NR-style recursive per axis: bits b0, b2, b4, b6 drive I and b1,
  b3, b5, b7 drive Q; with per-axis bits c0..c_{q-1} the amplitude is
  ``A(c0..) = (1 - 2 c0) * (2^(q-1) - A(c1..))`` and ``A(c) = 1 - 2c`` for one
  bit; normalised by 1/sqrt(2), 1/sqrt(10), 1/sqrt(42), 1/sqrt(170).
* AWGN: complex noise of variance sigma^2 per symbol (sigma^2 / 2 per axis).
"""
from __future__ import annotations

import numpy as np

from .basegraph import BaseGraph

CRC24_POLY = 0x864CFB  # x^24 + x^23 + x^18 + x^17 + x^14 + x^11 + x^10 + x^7 + x^6 + x^5 + x^4 + x^3 + x + 1
CRC24B_POLY = 0x800063  # x^24 + x^23 + x^6 + x^5 + x + 1 (per code block)
QAM_NORM = {2: np.sqrt(2.0), 4: np.sqrt(10.0), 6: np.sqrt(42.0), 8: np.sqrt(170.0)}


# --------------------------------------------------------------------------- CRC attach
def _xpow_mod_table(n: int, poly: int) -> np.ndarray:
    """rows[i] = bits of x^(24 + n - 1 - i) mod g, i.e. the parity contribution of message bit i."""
    cur = poly  # x^24 mod g: the low 24 bits of g
    vals = np.empty(n, dtype=np.int64)  # vals[j] = x^(24 + j) mod g
    for j in range(n):
        vals[j] = cur
        cur <<= 1  # multiply by x, then reduce
        if cur & (1 << 24):
            cur = (cur ^ (poly | (1 << 24))) & 0xFFFFFF
    # message bit i has weight x^(n - 1 - i); first output bit is the x^23 coefficient
    return ((vals[::-1, None] >> (23 - np.arange(24))[None, :]) & 1).astype(np.uint8)


_CRC_TABLE_CACHE: dict[tuple, np.ndarray] = {}


def crc24_attach(payload: np.ndarray, poly: int = CRC24_POLY) -> np.ndarray:
    """Append 24 CRC bits of generator ``poly`` to each row of ``payload`` (uint8 bits, shape (n, A))."""
    payload = np.asarray(payload, dtype=np.uint8)
    n_tb, A = payload.shape
    if (A, poly) not in _CRC_TABLE_CACHE:
        _CRC_TABLE_CACHE[(A, poly)] = _xpow_mod_table(A, poly).astype(np.float32)
    G = _CRC_TABLE_CACHE[(A, poly)]
    crc = (payload.astype(np.float32) @ G).astype(np.int64) & 1  # exact: sums <= A < 2^24
    return np.concatenate([payload, crc.astype(np.uint8)], axis=1)


# --------------------------------------------------------------------------- encoder
def _rot(x: np.ndarray, s: int) -> np.ndarray:
    """(P^s x)[..., k] = x[..., (k + s) mod Z]."""
    return np.roll(x, -s, axis=-1)


def encode(bg: BaseGraph, Z: int, info: np.ndarray, n_cols: int | None = None) -> np.ndarray:
    """Systematic QC encoding of a batch: info (B, kb*Z) bits -> codewords (B, n_cols*Z).

    Only the first ``n_cols`` columns are produced (default: all ``nb``);
    extension parity columns beyond that are never transmitted.
    """
    info = np.asarray(info, dtype=np.uint8)
    B = info.shape[0]
    kb, mc = bg.kb, bg.mc
    n_cols = bg.nb if n_cols is None else n_cols
    u = info.reshape(B, kb, Z)
    blocks = np.zeros((B, bg.nb, Z), dtype=np.uint8)
    blocks[:, :kb] = u
    rows = [bg.row_edges(r) for r in range(bg.mb)]
    lam = np.zeros((B, mc, Z), dtype=np.uint8)
    for r in range(mc):
        cols, V = rows[r]
        for c, v in zip(cols, V):
            if c < kb:
                lam[:, r] ^= _rot(u[:, c], int(v) % Z)
    r_mid = mc // 2
    p0 = np.bitwise_xor.reduce(lam, axis=1)
    blocks[:, kb] = p0
    if mc > 1:
        s_a = 1 % Z
        p = _rot(p0, s_a) ^ lam[:, 0]
        blocks[:, kb + 1] = p
        for i in range(1, mc - 1):
            p = lam[:, i] ^ p ^ (p0 if i == r_mid else 0)
            blocks[:, kb + i + 1] = p
    for r in range(mc, bg.mb):
        own = kb + r
        if own >= n_cols:
            break
        cols, V = rows[r]
        acc = np.zeros((B, Z), dtype=np.uint8)
        for c, v in zip(cols, V):
            if c != own:
                acc ^= _rot(blocks[:, c], int(v) % Z)
        blocks[:, own] = acc
    return blocks[:, :n_cols].reshape(B, n_cols * Z)


# --------------------------------------------------------------------------- rate match + QAM
def rate_match(bg: BaseGraph, Z: int, cw: np.ndarray, E: int, rv: int = 0) -> np.ndarray:
    """Redundancy version rv from a circular buffer of the codeword positions [t0, nb*Z): bit e is
    position t0 + ((k0 + e) mod Ncb), Ncb = nb*Z - t0, so a version that runs past the buffer's end
    continues from its start (at most two passes: E <= 2 Ncb)."""
    t0 = bg.t0(Z)
    ncb = bg.ncb(Z)
    k0 = bg.k0(Z, rv)
    if E > 2 * ncb:
        raise ValueError("E exceeds two passes over the circular buffer")
    pos = t0 + (k0 + np.arange(E)) % ncb
    if pos.max() >= cw.shape[1]:
        raise ValueError("the codeword does not reach the positions sent")
    return cw[:, pos]


def interleave(e: np.ndarray, Qm: int, enabled: bool = True) -> np.ndarray:
    """(B, E) -> (B, E/Qm, Qm): the Qm bits carried by each resource element."""
    B, E = e.shape
    n_re = E // Qm
    if enabled:
        return e.reshape(B, Qm, n_re).transpose(0, 2, 1)
    return e.reshape(B, n_re, Qm)


def _pam(bits: np.ndarray) -> np.ndarray:
    """Recursive Gray PAM amplitude for per-axis bits (..., q) (unnormalised)."""
    q = bits.shape[-1]
    sgn = 1.0 - 2.0 * bits.astype(np.float64)
    if q == 1:
        return sgn[..., 0]
    return sgn[..., 0] * (2.0 ** (q - 1) - _pam(bits[..., 1:]))


def qam_map(re_bits: np.ndarray) -> np.ndarray:
    """(..., Qm) bits per resource element -> complex128 unit-energy Gray QAM."""
    Qm = re_bits.shape[-1]
    I = _pam(re_bits[..., 0::2])
    Q = _pam(re_bits[..., 1::2])
    return (I + 1j * Q) / QAM_NORM[Qm]


def awgn(x: np.ndarray, sigma2: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """x + CN(0, sigma2); sigma2 broadcasts against x."""
    s = np.sqrt(np.asarray(sigma2, dtype=np.float64) / 2.0)
    n = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
    return x + s * n


def urllc_symbol() -> complex:
    """The URLLC data written over punctured REs: all-zero bits, QPSK."""
    return complex((1.0 + 1.0j) / np.sqrt(2.0))
