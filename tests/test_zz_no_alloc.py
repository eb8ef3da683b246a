"""decode_uniform_noalloc: the decode entry point that allocates no memory.

Some callers cannot call cudaMalloc -- code under a memory pool or budget
that may not grow once set up, a real-time receive loop where an
allocation's latency or failure is not acceptable, or a host application
that owns all device memory and hands the library only its buffers.
For them the library decodes code blocks of one shape using only the caller's
buffers and a fixed array compiled into the library.  This test calls that
entry point through the C-ABI (ctypes) and checks, on two calls in a row,
that its bits and status equal those of decode_batch on the same LLRs (the
tolerance is exact equality, as for every decoder comparison in these tests),
and that sizes beyond its fixed limit are refused before anything runs.

This file's name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2506_00167_gb300 import abi
from workload import large_fp32, mixed, tiny_fp32

from gpu_helpers import device_inputs, session_for

pytestmark = pytest.mark.gpu

LLR_DTYPE = {"f32": torch.float32, "i8": torch.int8, "i16": torch.int16}
SAT = {"f32": (0, 0), "i8": (63, 127), "i16": (1023, 32767)}


def _bg_struct(bg):
    keep = [np.ascontiguousarray(x, dtype=np.int16) for x in (bg.row, bg.col, bg.V)]
    p16 = ctypes.POINTER(ctypes.c_int16)
    s = abi.BaseGraphC(bg.mb, bg.nb, bg.kb, bg.mc, bg.n_punct_cols, keep[0].size,
                       keep[0].ctypes.data_as(p16), keep[1].ctypes.data_as(p16), keep[2].ctypes.data_as(p16))
    return s, keep


def _noalloc(bg, Z, E, n, mode, max_iter, et, llr, bits, status):
    lib = abi.load()
    s, keep = _bg_struct(bg)
    msg_sat, post_sat = SAT[mode]
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.decode_uniform_noalloc(ctypes.byref(s), Z, E, n, abi.MODES[mode], max_iter, int(et), 0.5, 1,
                                    msg_sat, post_sat, llr.data_ptr(), bits.data_ptr(), status.data_ptr(), stream)
    del keep
    return rc


def _uniform(w):
    """(base graph, Z, E) if every code block of w has one shape, with LLRs packed back to back."""
    c0 = w.cbs[0]
    for c in w.cbs:
        assert (c["bg"], c["Z"], c["E"]) == (c0["bg"], c0["Z"], c0["E"])
    bg, Z, t0, m_eff, n_eff = w.cb_geometry(0)
    assert np.array_equal(w.cbs["llr_offset"], np.arange(w.n_cb) * n_eff * Z)
    return bg, int(c0["Z"]), int(c0["E"])


CASES = [
    ("large", "f32"), ("large", "i8"), ("large", "i16"), ("tiny", "f32"), ("mixed_one_shape", "i8"),
    ("bg1_z16", "i8"), ("bg1_z16", "f32"),
]


def _workload(name):
    if name == "large":
        return large_fp32(n_cw=12, snr_points=(6, 8, 10))
    if name == "tiny":
        return tiny_fp32(n_per_point=16, ebn0_points=(1, 3))
    from workload.configs import TBSpec, build, default_bgs, es_n0_sigma2
    bgs = default_bgs()
    if name == "bg1_z16":  # two groups of 16 threads share each warp: the even-group launch form
        E = 2 * int(round(bgs[0].kb * 16 / (0.5 * 2)))
        specs = [TBSpec(i, 0, 16, 2, E, 1, float(es_n0_sigma2(s)), 0, 36) for i, s in enumerate([1.0, 3.0, 5.0] * 7)]
        return build("bg1_z16", bgs, specs, [36] * 21, [np.zeros((14, 36), bool)] * 21, seed=12)
    # one shape out of the mixed generator: BG2, Z = 64, rate 0.5, 64-QAM
    Z, Qm = 64, 6
    E = Qm * int(round(bgs[1].kb * Z / (0.5 * Qm)))
    specs = [TBSpec(i, 1, Z, Qm, E, 1, float(es_n0_sigma2(s)), 0, 48) for i, s in enumerate([6.0, 8.0, 10.0] * 3)]
    return build("one_shape", bgs, specs, [48] * 9, [np.zeros((14, 48), bool)] * 9, seed=11)


@pytest.mark.parametrize("name,mode", CASES)
def test_noalloc_matches_decode_batch_twice(name, mode):
    w = _workload(name)
    bg, Z, E = _uniform(w)
    mi = w.meta.get("max_iter", 10)
    et = bool(w.meta.get("early_term", 1))
    s = session_for(w, mode, max_iter=mi, early_term=et)
    b = s.batch(w.cbs)
    sym, mask = device_inputs(w)
    llr = torch.empty(b.info.llr_elems, dtype=LLR_DTYPE[mode], device="cuda")
    s.puncture_demap(b, sym, mask, llr)
    ref_bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
    ref_status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
    s.decode_batch(b, llr, ref_bits, ref_status)
    torch.cuda.synchronize()
    for call in range(2):
        bits = torch.full_like(ref_bits, -1)
        status = torch.full_like(ref_status, -1)
        rc = _noalloc(bg, Z, E, w.n_cb, mode, mi, et, llr, bits, status)
        assert rc == 0, abi.load().ldpc_last_error()
        torch.cuda.synchronize()
        assert torch.equal(bits, ref_bits), f"call {call}: bits differ"
        assert torch.equal(status, ref_status), f"call {call}: status differs"


def test_noalloc_rejects_sizes_beyond_its_limit():
    w = large_fp32(n_cw=2)
    bg, Z, E = _uniform(w)
    z = torch.zeros(16, dtype=torch.float32, device="cuda")
    zi = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = _noalloc(bg, Z, E, 32769, "f32", 10, True, z, zi, zi)
    assert rc == -1
    assert b"32768" in abi.load().ldpc_last_error()
    assert _noalloc(bg, Z, E, 0, "f32", 10, True, z, zi, zi) == 0


def _errors():
    v = ctypes.c_uint32(0xFFFFFFFF)
    rc = abi.load().decode_uniform_noalloc_errors(ctypes.byref(v), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, abi.load().ldpc_last_error()
    return v.value


def test_noalloc_reports_a_wait_that_runs_out():
    """The device error word: clean after a good call; a bounded bulk-copy wait that nothing completes
    sets LDPC_DEVERR_TMA_TIMEOUT there; reading clears it; the next call decodes normally."""
    w = large_fp32(n_cw=4, snr_points=(8,))
    bg, Z, E = _uniform(w)
    s = session_for(w, "i8")
    b = s.batch(w.cbs)
    sym, mask = device_inputs(w)
    llr = torch.empty(b.info.llr_elems, dtype=torch.int8, device="cuda")
    s.puncture_demap(b, sym, mask, llr)
    ref_bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
    ref_status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
    s.decode_batch(b, llr, ref_bits, ref_status)
    bits = torch.zeros_like(ref_bits)
    status = torch.zeros_like(ref_status)
    assert _noalloc(bg, Z, E, w.n_cb, "i8", 10, True, llr, bits, status) == 0
    assert _errors() == 0
    lib = abi.load()
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.decode_uniform_noalloc_wait_check(0, stream) == -1
    assert lib.decode_uniform_noalloc_wait_check(256, stream) == 0
    assert _errors() == 0x1          # LDPC_DEVERR_TMA_TIMEOUT
    assert _errors() == 0            # read and cleared
    bits.fill_(-1)
    status.fill_(-1)
    assert _noalloc(bg, Z, E, w.n_cb, "i8", 10, True, llr, bits, status) == 0
    torch.cuda.synchronize()
    assert torch.equal(bits, ref_bits) and torch.equal(status, ref_status)
    assert _errors() == 0

