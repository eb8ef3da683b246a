"""Layered offset-min-sum decoding of a QC-LDPC code (oracle; test infrastructure only).

The paper's receiver LDPC-decodes the flushed LLRs with a toolbox decoder
(Sec. VI-D "UE") and states neither algorithm nor parameters; this build fixes
layered offset min-sum.  Notation: the lifted check (l, k) of base row l
connects, through base edge (l, j) with column c_j and shift s_j = V mod Z,
to variable v_j(k) = c_j * Z + (k + s_j) mod Z.  With posterior L (initially
the channel LLRs) and check-to-variable messages R (initially 0), each
iteration runs the rows l = 0 .. m_eff-1 in order and, for all k at once:

    Q_j   = L[v_j] - R[l, j, k]                         (variable-to-check)
    sgn_j = [Q_j < 0]      (0 counts as positive)
    m1, m2, j* = smallest |Q_j|, second smallest, first index of the smallest
    R'_j  = (-1)^(XOR_{i != j} sgn_i) * max((m2 if j == j* else m1) - beta, 0)
    L[v_j] = Q_j + R'_j ;  R[l, j, k] = R'_j

After every full iteration (never before the first) the hard decision
c_v = [L_v < 0] is tested against the m_eff decoded rows; with early
termination on, a code block whose syndrome is zero stops there.  A code
block that carries its own CRC (the last 24 of its K information bits, see
``crc``) also stops when its K hard-decided information bits pass that CRC
(CRC-aided early termination, the usual exit of NR receivers; the paper's
toolbox decoder is not described further, Sec. VI-D "UE").  Output: the
K = kb * Z information bits (columns 0 .. kb-1), the iterations run, whether
the final syndrome was zero and, for a block with a CRC, whether its final
information bits pass it.

Integer modes (exact int64 arithmetic, then saturation):
INT8  Q = sat127(L - R); |Q| clamped to 63 before the minimum; offset 1;
      L = sat127(Q + R').
INT16 Q, L saturate at +-32767; |Q| clamped to 1023; offset 1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import crc
from .demap import bg_geometry, rv_of


@dataclass(frozen=True)
class FloatArith:
    beta: float = 0.5
    dtype: type = np.float64

    def prep(self, x):
        return np.asarray(x, dtype=self.dtype)

    def post(self, x):
        return x

    def msg(self, a):
        return a

    def big(self):
        return self.dtype(np.inf)


@dataclass(frozen=True)
class IntArith:
    beta: int = 1
    msg_sat: int = 63
    post_sat: int = 127

    def prep(self, x):
        return np.asarray(x, dtype=np.int64)

    def post(self, x):
        return np.clip(x, -self.post_sat, self.post_sat)

    def msg(self, a):
        return np.minimum(a, self.msg_sat)

    def big(self):
        return np.int64(self.msg_sat + 1)


INT8 = IntArith(1, 63, 127)
INT16 = IntArith(1, 1023, 32767)
F64 = FloatArith(0.5, np.float64)
F32 = FloatArith(0.5, np.float32)


def _rows(bg, Z, m_eff):
    out = []
    for l in range(m_eff):
        sel = bg.row == l
        cols = bg.col[sel].astype(np.int64)
        s = bg.V[sel].astype(np.int64) % Z
        order = np.argsort(cols, kind="stable")
        cols, s = cols[order], s[order]
        vidx = (np.arange(Z)[None, :] + s[:, None]) % Z     # (deg, Z)
        out.append((cols, vidx))
    return out


def _syndrome_ok(L, rows):
    hard = L < 0
    ok = np.ones(L.shape[0], dtype=bool)
    for cols, vidx in rows:
        par = np.bitwise_xor.reduce(hard[:, cols[:, None], vidx], axis=1)  # (B, Z)
        ok &= ~par.any(axis=1)
    return ok


def layered_oms(llr, bg, Z, m_eff, max_iter, early_term, arith=F64, return_L=False, cb_crc=None,
                with_crc=False):
    """Decode a batch of code blocks of one shape.

    llr: (B, n_eff*Z) channel LLRs (int for IntArith); ``cb_crc``: bool (B,),
    True for a block whose information bits end in a CRC-24 (0x800063).
    Returns (bits uint8 (B, kb*Z), iters int (B,), ok bool (B,)[, crc_ok bool
    (B,) with ``with_crc``][, L final (B, n_eff*Z)]).
    """
    kb = bg.kb
    n_eff = kb + m_eff
    llr = arith.prep(llr)
    B = llr.shape[0]
    assert llr.shape[1] == n_eff * Z
    rows = _rows(bg, Z, m_eff)
    if any(c.size < 2 for c, _ in rows):
        raise ValueError("every decoded row needs degree >= 2")

    L = llr.reshape(B, n_eff, Z).copy()
    R = [np.zeros((B, c.size, Z), dtype=L.dtype) for c, _ in rows]
    beta = arith.prep(arith.beta) if isinstance(arith, IntArith) else L.dtype.type(arith.beta)
    zero = L.dtype.type(0)

    bits = np.zeros((B, kb * Z), dtype=np.uint8)
    iters = np.full(B, max_iter, dtype=np.int64)
    ok = np.zeros(B, dtype=bool)
    crc_ok = np.zeros(B, dtype=bool)
    flag = np.zeros(B, dtype=bool) if cb_crc is None else np.asarray(cb_crc, dtype=bool).copy()
    L_out = np.zeros((B, n_eff, Z), dtype=L.dtype)
    active = np.arange(B)

    for it in range(1, max_iter + 1):
        for l, (cols, vidx) in enumerate(rows):
            deg = cols.size
            Q = arith.post(L[:, cols[:, None], vidx] - R[l])          # (b, deg, Z)
            mag = arith.msg(np.abs(Q))
            neg = Q < 0
            j_star = np.argmin(mag, axis=1)                            # first occurrence
            m1 = np.take_along_axis(mag, j_star[:, None, :], axis=1)[:, 0, :]
            masked = mag.copy()
            np.put_along_axis(masked, j_star[:, None, :], arith.big(), axis=1)
            m2 = masked.min(axis=1)
            parity = np.bitwise_xor.reduce(neg, axis=1)                # (b, Z)
            j = np.arange(deg)[None, :, None]
            excl = np.where(j == j_star[:, None, :], m2[:, None, :], m1[:, None, :])
            Rmag = np.maximum(excl - beta, zero)
            Rn = np.where(neg ^ parity[:, None, :], -Rmag, Rmag)
            L[:, cols[:, None], vidx] = arith.post(Q + Rn)
            R[l] = Rn
        last = it == max_iter
        if early_term or last:
            s_ok = _syndrome_ok(L, rows)
            c_ok = np.zeros_like(s_ok)
            if flag.any():
                hard = (L[flag, :kb, :] < 0).reshape(int(flag.sum()), kb * Z).astype(np.uint8)
                c_ok[flag] = crc.cb_ok(hard).astype(bool)
            done = (s_ok | c_ok) if early_term else np.zeros_like(s_ok)
            if last:
                done = np.ones_like(s_ok)
            if done.any():
                g = active[done]
                bits[g] = (L[done, :kb, :] < 0).reshape(done.sum(), kb * Z).astype(np.uint8)
                iters[g] = it
                ok[g] = s_ok[done]
                crc_ok[g] = c_ok[done]
                L_out[g] = L[done]
                keep = ~done
                active = active[keep]
                L = L[keep]
                flag = flag[keep]
                R = [r[keep] for r in R]
            if active.size == 0:
                break
    out = (bits, iters, ok) + ((crc_ok,) if with_crc else ())
    if return_L:
        return out + (L_out.reshape(B, n_eff * Z),)
    return out


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """(n, 32m) bits -> (n, m) uint32 with bit i at bit i % 32 of word i // 32."""
    n, Lb = bits.shape
    b = bits.reshape(n, Lb // 32, 32).astype(np.uint64)
    return (b << np.arange(32, dtype=np.uint64)).sum(axis=2).astype(np.uint32)


def status_word(iters, ok, crc_ok=None):
    """Status per code block: iterations in bits 0..15, syndrome-zero flag in bit 16, and in bit 17
    the flag of a block with its own CRC whose final information bits pass it."""
    st = np.asarray(iters, dtype=np.int64) | (np.asarray(ok, dtype=np.int64) << 16)
    if crc_ok is not None:
        st |= np.asarray(crc_ok, dtype=np.int64) << 17
    return st.astype(np.int32)


def decode_workload(w, llr, max_iter, early_term, arith=F64, cb_index=None, return_L=False):
    """Decode every (or the listed) code block of workload ``w`` from the LLR buffer ``llr``.

    Returns (bits words uint32 (w.bits_words,), status int32 (n_cb,)) and, with
    ``return_L``, the final posterior buffer shaped like ``llr``.
    """
    idx = np.arange(w.n_cb) if cb_index is None else np.asarray(cb_index)
    words = np.zeros(w.bits_words, dtype=np.uint32)
    status = np.zeros(w.n_cb, dtype=np.int32)
    Lbuf = np.zeros(w.llr_len, dtype=np.float64 if isinstance(arith, FloatArith) else np.int64) \
        if return_L else None
    groups: dict = {}
    for i in idx:
        c = w.cbs[i]
        bg = w.bgs[int(c["bg"])]
        Z, E = int(c["Z"]), int(c["E"])
        _, m_eff, n_eff = bg_geometry(bg, Z, E, rv_of(c))
        groups.setdefault((int(c["bg"]), Z, m_eff), []).append(int(i))
    for (b, Z, m_eff), members in groups.items():
        bg = w.bgs[b]
        n = (bg.kb + m_eff) * Z
        x = np.stack([llr[int(w.cbs[i]["llr_offset"]):int(w.cbs[i]["llr_offset"]) + n] for i in members])
        flags = np.array([int(w.cbs[i]["flags"]) & 1 for i in members], dtype=bool)
        res = layered_oms(x, bg, Z, m_eff, max_iter, early_term, arith, return_L=return_L, cb_crc=flags,
                          with_crc=True)
        bits, iters, ok, c_ok = res[:4]
        pw = pack_bits(bits)
        st = status_word(iters, ok, c_ok)
        for r, i in enumerate(members):
            o = int(w.cbs[i]["bits_word_offset"])
            words[o:o + pw.shape[1]] = pw[r]
            status[i] = st[r]
            if return_L:
                lo = int(w.cbs[i]["llr_offset"])
                Lbuf[lo:lo + n] = res[4][r]
    if return_L:
        return words, status, Lbuf
    return words, status
