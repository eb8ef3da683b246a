"""CRC-24 over a transport block (oracle; test infrastructure only).

The paper sets d_e from a bitwise comparison of the CRC bits recovered after
decoding with those attached at the transmitter (Sec. VI-D "UE Feedback";
Sec. III-B defines d_e).  It names no polynomial; this build uses generator
g(x) = x^24 + x^23 + x^18 + x^17 + x^14 + x^11 + x^10 + x^7 + x^6 + x^5 + x^4
+ x^3 + x + 1 (0x864CFB), register starting at 0, first bit = highest-degree
coefficient, no reflection, no final xor.  Comparing the received CRC with
the one recomputed from the received payload is the same test as asking
whether the whole received (A + 24)-bit word is a multiple of g(x), which is
what ``tb_ok`` checks.
"""
from __future__ import annotations

import numpy as np

POLY = 0x864CFB
MASK = 0xFFFFFF


def remainder_bitwise(bits: np.ndarray) -> np.ndarray:
    """M(x) * x^24 mod g(x) by long division, one bit at a time.

    ``bits``: uint8 array (n, L) (or (L,)); returns int64 (n,) remainders.
    """
    b = np.atleast_2d(np.asarray(bits, dtype=np.int64))
    reg = np.zeros(b.shape[0], dtype=np.int64)
    for i in range(b.shape[1]):
        fb = ((reg >> 23) & 1) ^ b[:, i]
        reg = (reg << 1) & MASK
        reg ^= fb * POLY
    return reg


def _byte_table() -> np.ndarray:
    t = np.zeros(256, dtype=np.int64)
    for v in range(256):
        r = v << 16
        for _ in range(8):
            r = ((r << 1) ^ POLY) & MASK if r & 0x800000 else (r << 1) & MASK
        t[v] = r
    return t


_TABLE = _byte_table()


def remainder_table(bits: np.ndarray) -> np.ndarray:
    """Same remainder, eight bits per step through a 256-entry table (L % 8 == 0)."""
    b = np.atleast_2d(np.asarray(bits, dtype=np.int64))
    n, L = b.shape
    if L % 8:
        raise ValueError("table CRC wants a whole number of bytes")
    by = (b.reshape(n, L // 8, 8) << np.arange(7, -1, -1)).sum(axis=2)
    reg = np.zeros(n, dtype=np.int64)
    for i in range(L // 8):
        reg = ((reg << 8) & MASK) ^ _TABLE[((reg >> 16) ^ by[:, i]) & 0xFF]
    return reg


def crc_bits(payload: np.ndarray) -> np.ndarray:
    """The 24 CRC bits for ``payload`` (n, A), first bit = x^23 coefficient."""
    r = remainder_bitwise(payload)
    return ((r[:, None] >> (23 - np.arange(24))[None, :]) & 1).astype(np.uint8)


def tb_ok(tb_bits: np.ndarray) -> np.ndarray:
    """d_e: 1 where the received (A + 24) bits leave remainder 0, else 0."""
    return (remainder_bitwise(tb_bits) == 0).astype(np.uint8)
