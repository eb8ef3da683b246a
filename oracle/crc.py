"""CRC-24 over transport blocks and code blocks (oracle; test infrastructure only).

The paper sets d_e from a bitwise comparison of the CRC bits recovered after
decoding with those attached at the transmitter (Sec. VI-D "UE Feedback";
Sec. III-B defines d_e).  It names no polynomial; this build uses generator
g_A(x) = x^24 + x^23 + x^18 + x^17 + x^14 + x^11 + x^10 + x^7 + x^6 + x^5 + x^4
+ x^3 + x + 1 (0x864CFB), register starting at 0, first bit = highest-degree
coefficient, no reflection, no final xor.  Comparing the received CRC with
the one recomputed from the received payload is the same test as asking
whether the whole received (A + 24)-bit word is a multiple of g_A(x), which is
what ``tb_ok`` checks.

Segmented transport blocks (more than one code block) may also carry a CRC
per code block, NR style: the last 24 of a code block's K bits are the CRC of
its first K - 24 under g_B(x) = x^24 + x^23 + x^6 + x^5 + x + 1 (0x800063),
same conventions.  The paper's Tx chain appends CRC bits without saying
where (Sec. VI-A, "Tx Signal Processing"); the per-code-block CRC is this
build's reading of a segmented NR transport block.  ``cb_ok`` checks it.
"""
from __future__ import annotations

import numpy as np

POLY = 0x864CFB    # g_A: one per transport block
POLY_B = 0x800063  # g_B: one per code block of a segmented transport block
MASK = 0xFFFFFF


def remainder_bitwise(bits: np.ndarray, poly: int = POLY) -> np.ndarray:
    """M(x) * x^24 mod g(x) by long division, one bit at a time.

    ``bits``: uint8 array (n, L) (or (L,)); returns int64 (n,) remainders.
    """
    b = np.atleast_2d(np.asarray(bits, dtype=np.int64))
    reg = np.zeros(b.shape[0], dtype=np.int64)
    for i in range(b.shape[1]):
        fb = ((reg >> 23) & 1) ^ b[:, i]
        reg = (reg << 1) & MASK
        reg ^= fb * poly
    return reg


def _byte_table(poly: int) -> np.ndarray:
    t = np.zeros(256, dtype=np.int64)
    for v in range(256):
        r = v << 16
        for _ in range(8):
            r = ((r << 1) ^ poly) & MASK if r & 0x800000 else (r << 1) & MASK
        t[v] = r
    return t


_TABLES = {POLY: _byte_table(POLY), POLY_B: _byte_table(POLY_B)}


def remainder_table(bits: np.ndarray, poly: int = POLY) -> np.ndarray:
    """Same remainder, eight bits per step through a 256-entry table (L % 8 == 0)."""
    b = np.atleast_2d(np.asarray(bits, dtype=np.int64))
    n, L = b.shape
    if L % 8:
        raise ValueError("table CRC wants a whole number of bytes")
    table = _TABLES[poly] if poly in _TABLES else _byte_table(poly)
    by = (b.reshape(n, L // 8, 8) << np.arange(7, -1, -1)).sum(axis=2)
    reg = np.zeros(n, dtype=np.int64)
    for i in range(L // 8):
        reg = ((reg << 8) & MASK) ^ table[((reg >> 16) ^ by[:, i]) & 0xFF]
    return reg


def crc_bits(payload: np.ndarray, poly: int = POLY) -> np.ndarray:
    """The 24 CRC bits for ``payload`` (n, A), first bit = x^23 coefficient."""
    r = remainder_bitwise(payload, poly)
    return ((r[:, None] >> (23 - np.arange(24))[None, :]) & 1).astype(np.uint8)


def tb_ok(tb_bits: np.ndarray) -> np.ndarray:
    """d_e: 1 where the received (A + 24) bits leave remainder 0 under g_A, else 0."""
    return (remainder_bitwise(tb_bits) == 0).astype(np.uint8)


def cb_ok(cb_bits: np.ndarray) -> np.ndarray:
    """1 where a code block's K received bits leave remainder 0 under g_B, else 0."""
    b = np.atleast_2d(np.asarray(cb_bits))
    rem = remainder_table(b, POLY_B) if b.shape[1] % 8 == 0 else remainder_bitwise(b, POLY_B)
    return (rem == 0).astype(np.uint8)
