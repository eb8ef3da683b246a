"""The whole receive path on the CPU (oracle; test infrastructure only).

puncture flushing + max-log demap (``demap``) -> layered offset min-sum
(``decoder``) -> TB CRC-24, goodput and reward (``goodput``), in the order of
Sec. VI-D "UE".  Used by the parity tests and by the benchmark's timed CPU
baseline.
"""
from __future__ import annotations

import numpy as np

from . import decoder, demap, goodput

MODES = {
    "f64": (decoder.F64, None, None),
    "f32": (decoder.F32, None, None),
    "i8": (decoder.INT8, 4.0, 63),
    "i16": (decoder.INT16, 4.0, 1023),
}


def run(w, mode="f64", max_iter=10, early_term=True, cb_index=None):
    """Returns dict(llr, words, status, d, goodput_bits, goodput_sc, reward)."""
    arith, scale, sat = MODES[mode]
    llr = demap.demap_workload(w, cb_index)
    if scale is not None:
        llr_in = demap.quantise(llr, scale, sat)
    else:
        llr_in = llr.astype(arith.dtype)
    words, status = decoder.decode_workload(w, llr_in, max_iter, early_term, arith, cb_index)
    out = dict(llr=llr_in, words=words, status=status)
    if cb_index is None:
        d, gb, gs, r = goodput.tb_crc_goodput(w, words)
        out.update(d=d, goodput_bits=gb, goodput_sc=gs, reward=r)
    return out


def block_errors(w, words) -> np.ndarray:
    """Per code block: 1 where the decoded information bits differ from those sent."""
    err = np.zeros(w.n_cb, dtype=np.uint8)
    for i, c in enumerate(w.cbs):
        K = w.bgs[int(c["bg"])].kb * int(c["Z"])
        o = int(c["bits_word_offset"])
        err[i] = np.any(words[o:o + K // 32] != w.info_words[o:o + K // 32])
    return err
