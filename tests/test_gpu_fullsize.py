"""GPU parity at the benchmark's full sizes, in the launch configuration bench.py times.

The large workload (4096 BG1-shaped Z=384 code blocks) and the mixed workload (512 slots, ~18,000 code
blocks of ten shapes, one persistent launch), with the autotuned tiles bench.py applies.  The oracle
cannot decode those batches in seconds, so it checks a seeded sample one by one: the sampled blocks'
LLRs are replaced by the oracle's own before the full-size decode (each block's decode depends on its
LLRs only), and their bits, status words and TB outcomes must equal the oracle's.  Properties that hold
at any size (eq. 1 and eq. 2 from the GPU's own d_e, iteration bounds) cover the rest.
"""
import numpy as np
import pytest
import torch

import bench
from oracle import decoder as odec
from oracle import demap as odemap
from oracle import goodput as ogood
from paper_2506_00167_gb300 import Session

from gpu_helpers import LLR_NP, SAT, device_inputs, to_np_u32

pytestmark = pytest.mark.gpu

ARITH = {"f32": odec.F32, "i8": odec.INT8}


def _oracle_llr(w, mode, cb_index):
    llr = odemap.demap_workload(w, cb_index=cb_index)
    return llr.astype(np.float32) if mode == "f32" else odemap.quantise(llr, 4.0, 63)


def _segments(w, cb_index):
    for i in cb_index:
        bg, Z, t0, m_eff, n_eff = w.cb_geometry(int(i))
        o = int(w.cbs[int(i)]["llr_offset"])
        yield int(i), o, o + n_eff * Z


@pytest.mark.parametrize("name,mode,cb_crc", [("large", "f32", False), ("large", "i8", False),
                                              ("mixed", "i8", False), ("mixed", "i8", True)])
def test_full_size_sampled_parity(name, mode, cb_crc):
    w = bench.make_workload(name, cb_crc=cb_crc)
    mi, et = w.meta["max_iter"], bool(w.meta["early_term"])
    s = Session(w.bgs, w.z_set, mode=mode, max_iter=mi, early_term=et, sat=SAT[mode])
    bench.apply_tiles(s, w, mode, "auto", 1)
    b = s.batch(w.cbs, w.tbs, w.slot_N)
    sym, mask = device_inputs(w)
    out = b.alloc_outputs()
    s.run(b, sym, mask, out)  # one whole step, as timed
    torch.cuda.synchronize()
    assert s.device_errors() == 0

    # ---- a seeded sample of TBs (all their code blocks)
    rng = np.random.default_rng(1234)
    tbs = np.sort(rng.choice(w.n_tb, size=12 if name == "mixed" else 24, replace=False))
    cbs = np.concatenate([np.arange(int(w.tbs[t]["first_cb"]), int(w.tbs[t]["first_cb"]) + int(w.tbs[t]["n_cb"]))
                          for t in tbs])

    # demap: the full-size step's LLRs of the sampled blocks against the float64 oracle
    got = out["llr"].cpu().numpy()
    want64 = odemap.demap_workload(w, cb_index=cbs)
    for i, lo, hi in _segments(w, cbs):
        g = got[lo:hi].astype(np.float64)
        if mode == "f32":
            assert np.all(np.abs(g - want64[lo:hi]) <= 1e-4 * np.maximum(np.abs(want64[lo:hi]), 1.0)), i
        else:
            q = odemap.quantise(want64[lo:hi], 4.0, 63)
            assert np.abs(g - q).max() <= 1, i

    # decode + CRC at full size with the sampled blocks' LLRs taken from the oracle
    want_llr = _oracle_llr(w, mode, cbs)
    llr = out["llr"].clone()
    for i, lo, hi in _segments(w, cbs):
        llr[lo:hi] = torch.from_numpy(want_llr[lo:hi].astype(LLR_NP[mode])).cuda()
    s.decode_batch(b, llr, out["bits"], out["status"])
    s.tb_crc_goodput(b, out["bits"], out["d"], out["goodput_bits"], out["goodput_sc"], out["reward"])
    torch.cuda.synchronize()
    want_bits, want_status = odec.decode_workload(w, want_llr, mi, et, ARITH[mode], cb_index=cbs)
    bits = to_np_u32(out["bits"])
    status = out["status"].cpu().numpy()
    for i in cbs:
        c = w.cbs[int(i)]
        K = w.bgs[int(c["bg"])].kb * int(c["Z"])
        o = int(c["bits_word_offset"])
        assert np.array_equal(bits[o:o + K // 32], want_bits[o:o + K // 32]), int(i)
        assert status[int(i)] == want_status[int(i)], int(i)
    d_gpu = out["d"].cpu().numpy()[:w.n_tb]
    d_want, _, _, _ = ogood.tb_crc_goodput(w, want_bits, tb_index=tbs)
    assert np.array_equal(d_gpu[tbs], d_want[tbs])

    # properties at the full size: iteration bounds, eq. 1 and eq. 2 from the GPU's own d_e
    it = status & 0xFFFF
    assert it.min() >= 1 and it.max() <= mi
    n_sc = w.tbs["n_sc"].astype(np.int64)
    slot = w.tbs["slot"].astype(np.int64)
    gs = np.bincount(slot, weights=d_gpu * n_sc, minlength=w.n_slots).astype(np.int64)
    fail = np.bincount(slot, weights=(1 - d_gpu.astype(np.int64)) * n_sc, minlength=w.n_slots)
    assert np.array_equal(out["goodput_sc"].cpu().numpy()[:w.n_slots].astype(np.int64), gs)
    r = out["reward"].cpu().numpy()[:w.n_slots].astype(np.float64)
    assert np.allclose(r, -fail / w.slot_N, rtol=2.0 ** -22, atol=0)
    gb = np.bincount(slot, weights=d_gpu * w.tbs["payload_bits"].astype(np.int64), minlength=w.n_slots)
    assert np.array_equal(out["goodput_bits"].cpu().numpy()[:w.n_slots].astype(np.int64), gb.astype(np.int64))
    assert s.device_errors() == 0
