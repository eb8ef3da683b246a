"""Precision on the GPU against the float64 oracle: BLER inside the oracle's 95 % Wilson interval."""
import numpy as np
import pytest
import torch

from oracle import path as opath
from oracle.stats import wilson
from workload import large_fp32

from gpu_helpers import batch_for, device_inputs, session_for

pytestmark = pytest.mark.gpu


def test_fp32_and_int16_bler_inside_oracle_interval():
    # 7.5 dB Es/N0 sits in the waterfall of this code (BLER ~ 0.4), where a
    # precision loss would show first
    w = large_fp32(n_cw=192, snr_points=(7.5,), seed=71)
    ref = opath.run(w, "f64", 10, True)
    err_ref = opath.block_errors(w, ref["words"])
    lo, hi = wilson(int(err_ref.sum()), w.n_cb)
    assert 0.05 < err_ref.mean() < 0.95
    sym, mask = device_inputs(w)
    for mode in ["f32", "i16"]:
        s = session_for(w, mode)
        b = batch_for(s, w)
        out = s.run(b, sym, mask, b.alloc_outputs())
        torch.cuda.synchronize()
        err = opath.block_errors(w, out["bits"].cpu().numpy().view(np.uint32))
        assert lo <= err.mean() <= hi, (mode, err.mean(), lo, hi)
        if mode == "f32":
            # same algorithm, float32 vs float64 rounding: block by block the
            # outcomes agree almost always (INT16 runs a 1-LSB = 0.25 offset, a
            # different algorithm, compared by BLER only)
            assert np.mean(err == err_ref) >= 0.97


def test_int8_bler_of_the_mixed_shapes_inside_the_oracle_int8_interval():
    """INT8 end to end on shapes of the mixed workload (BG1/BG2-shaped, Z = 32/64, rates 0.3-0.9,
    QPSK..256-QAM; the served stream's URLLC puncturing on shared slot grids) at the waterfall: the GPU's
    float32 demap + quantisation + INT8 decode against the oracle's float64 demap + quantisation + integer
    decode.  The decoders are bit-exact on equal inputs, so this checks the quantised demap end to end:
    the GPU block error rate lies inside the 95 % Wilson interval of the oracle's (oracle: 0.385)."""
    from workload.serving import codebook_bitmaps, served_workload, slot_stream, tb_pool
    pool = tb_pool(80, seed=73, max_cb=4, zs=(32, 64), snr_range_db=(-1.0, 1.0))
    st = slot_stream(6, pool.tbs["n_sc"], n_ue=24, tb_per_slot=1.0, seed=74)
    w = served_workload(pool, st["pool"], st["pattern"], st["grid_sc"], codebook_bitmaps())
    ref = opath.run(w, "i8", 10, True)
    err_ref = opath.block_errors(w, ref["words"])
    lo, hi = wilson(int(err_ref.sum()), w.n_cb)
    assert 0.05 < err_ref.mean() < 0.95, err_ref.mean()
    sym, mask = device_inputs(w)
    s = session_for(w, "i8")
    b = batch_for(s, w)
    out = s.run(b, sym, mask, b.alloc_outputs())
    torch.cuda.synchronize()
    err = opath.block_errors(w, out["bits"].cpu().numpy().view(np.uint32))
    assert lo <= err.mean() <= hi, (err.mean(), lo, hi)
    assert np.mean(err == err_ref) >= 0.97
