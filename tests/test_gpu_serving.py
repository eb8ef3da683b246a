"""Continuous-batching decode service (GPU): same result alone and in the mix, admission, idle relaunch."""
import time

import numpy as np
import pytest
import torch

from paper_2506_00167_gb300 import LdpcError, Server, abi
from workload.configs import subset
from workload.serving import pool_bytes, tb_pool, tb_records

from gpu_helpers import device_inputs, session_for

pytestmark = pytest.mark.gpu

# INT8 decode forms of the service: (paired, pair_threshold, which item counters must be nonzero).
# "auto" with a threshold of 4 items: a burst starts single and pairs once 4 items are in flight.
FORMS = [("auto", 4, ("items_single", "items_paired")), (True, 0, ("items_paired",)),
         (False, 0, ("items_single",))]
FORM_IDS = ["auto", "paired", "single"]


def _check_forms(srv, must):
    st = srv.stats()
    for k in ("items_single", "items_paired"):
        assert (st[k] > 0) == (k in must), st


@pytest.fixture(scope="module")
def pool():
    w = tb_pool(40, seed=7)
    raw, mask_base = pool_bytes(w)
    host = torch.from_numpy(raw).pin_memory()
    return w, host, mask_base


def _tb_words(w, t):
    tb = w.tbs[t]
    c = w.cbs[int(tb["first_cb"])]
    return int(tb["n_cb"]) * w.bgs[int(c["bg"])].kb * int(c["Z"]) // 32


def _wait(srv, n, timeout=20.0):
    got = []
    t0 = time.time()
    while sum(g.size for g in got) < n:
        got.append(srv.poll())
        assert time.time() - t0 < timeout, "service did not complete in time"
    return np.concatenate(got)


def _batch_reference(w, idx, mode="i8"):
    """The same TBs through the batch path (puncture_demap + decode_batch + tb_crc_goodput): d_e, bits and
    the most iterations of any code block, per TB."""
    sub = subset(w, idx)
    s = session_for(sub, mode)
    b = s.batch(sub.cbs, sub.tbs, sub.slot_N)
    sym, mask = device_inputs(sub)
    out = s.run(b, sym, mask, b.alloc_outputs())
    torch.cuda.synchronize()
    bits = out["bits"].cpu().numpy().view(np.uint32)
    status = out["status"].cpu().numpy()
    per_tb = []
    iters = []
    for t in range(sub.n_tb):
        first, n = int(sub.tbs[t]["first_cb"]), int(sub.tbs[t]["n_cb"])
        c = sub.cbs[first]
        o = int(c["bits_word_offset"])
        per_tb.append(bits[o:o + _tb_words(sub, t)].copy())
        iters.append(int((status[first:first + n] & 0xFFFF).max()))
    return out["d"].cpu().numpy()[:sub.n_tb], per_tb, iters


def test_result_is_the_same_alone_and_in_the_mix(pool):
    w, host, mask_base = pool
    n = w.n_tb
    words = [_tb_words(w, t) for t in range(n)]
    offs = np.concatenate([[0], np.cumsum(words)]).astype(np.int64)
    res = torch.zeros(2 * int(offs[-1]), dtype=torch.int32).pin_memory()
    s = session_for(w, "i8")
    srv = Server(s, host, res, arena_bytes=1 << 26, max_inflight=256)
    alone = [0, 3, 7, 11]
    # alone: one request at a time on an idle service
    d_alone = {}
    for t in alone:
        rec = tb_records(w, mask_base, abi.SERVE_TB_NP, pool_index=[t], tags=[t], result_offsets=[4 * offs[t]])
        assert srv.submit(rec) == 1
        done = _wait(srv, 1)
        assert int(done["tag"][0]) == t
        d_alone[t] = int(done["d"][0])
    bits_alone = {t: res[offs[t]:offs[t + 1]].numpy().view(np.uint32).copy() for t in alone}
    # in the mix: every TB arrives together (results into the second half of the result pool)
    base = int(offs[-1])
    recs = tb_records(w, mask_base, abi.SERVE_TB_NP, tags=np.arange(n), result_offsets=4 * (base + offs[:-1]))
    done = srv.replay(recs, np.zeros(n, np.int64), timeout_ms=20000)
    assert sorted(done["tag"].tolist()) == list(range(n))
    d_mix = {int(r["tag"]): int(r["d"]) for r in done}
    for t in alone:
        assert d_mix[t] == d_alone[t]
        assert np.array_equal(res[base + offs[t]:base + offs[t + 1]].numpy().view(np.uint32), bits_alone[t])
    # and both equal the batch path bit for bit, iteration counts included
    d_ref, bits_ref, it_ref = _batch_reference(w, range(n))
    it_mix = {int(r["tag"]): int(r["max_iters"]) for r in done}
    for t in range(n):
        assert d_mix[t] == int(d_ref[t]), t
        assert it_mix[t] == it_ref[t], t
        assert np.array_equal(res[base + offs[t]:base + offs[t + 1]].numpy().view(np.uint32), bits_ref[t]), t
    assert 0 < sum(d_mix.values()) <= n
    lat = (done["t_complete_ns"] - done["t_submit_ns"]) / 1e3
    assert np.all(lat > 0)
    srv.stop()


def test_admission_waits_for_memory(pool):
    w, host, mask_base = pool
    s = session_for(w, "i8")
    need = [_tb_words(w, t) + int(w.tbs[t]["n_cb"]) for t in range(3)]
    srv = Server(s, host, None, arena_bytes=4 * (need[0] + need[1]), max_inflight=64)
    recs = tb_records(w, mask_base, abi.SERVE_TB_NP, pool_index=[0, 1, 2], tags=[0, 1, 2])
    assert srv.submit(recs) == 2          # the third does not fit the arena yet
    done = _wait(srv, 2)
    assert sorted(done["tag"].tolist()) == [0, 1]
    assert srv.submit(recs[2:]) == 1      # admitted once the first two freed their space
    assert _wait(srv, 1)["tag"][0] == 2
    srv.stop()


def test_idle_loop_is_relaunched_and_bad_requests_rejected(pool):
    w, host, mask_base = pool
    s = session_for(w, "i8")
    srv = Server(s, host, None, arena_bytes=1 << 24, max_inflight=16, idle_timeout_us=2000)
    rec = tb_records(w, mask_base, abi.SERVE_TB_NP, pool_index=[5], tags=[1])
    assert srv.submit(rec) == 1
    _wait(srv, 1)
    time.sleep(0.05)                      # the device loop idles out meanwhile
    rec["tag"] = 2
    assert srv.submit(rec) == 1
    assert _wait(srv, 1)["tag"][0] == 2
    bad = rec.copy()
    bad["Z"] = 48
    with pytest.raises(LdpcError, match="EINVAL"):
        srv.submit(bad)
    bad = rec.copy()
    bad["sym_offset"] = host.numel()
    with pytest.raises(LdpcError, match="host pool"):
        srv.submit(bad)
    srv.stop()


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_repetition_blocks_through_the_service_match_the_batch_path(form):
    """Code blocks whose rate matching wraps the circular buffer: the service's fused demap combines the
    repeated LLRs like the batch demapper, bit for bit."""
    from workload.configs import repetition
    w = repetition(n_per_shape=4, seed=13)
    raw, mask_base = pool_bytes(w)
    host = torch.from_numpy(raw).pin_memory()
    n = w.n_tb
    words = [_tb_words(w, t) for t in range(n)]
    offs = np.concatenate([[0], np.cumsum(words)]).astype(np.int64)
    res = torch.zeros(int(offs[-1]), dtype=torch.int32).pin_memory()
    s = session_for(w, "i8")
    srv = Server(s, host, res, arena_bytes=1 << 24, max_inflight=64, paired=form[0], pair_threshold=form[1])
    try:
        recs = tb_records(w, mask_base, abi.SERVE_TB_NP, tags=np.arange(n), result_offsets=4 * offs[:-1])
        done = srv.replay(recs, np.zeros(n, np.int64), timeout_ms=20000)
        assert sorted(done["tag"].tolist()) == list(range(n))
        _check_forms(srv, form[2])
        d_ref, bits_ref, _ = _batch_reference(w, range(n))
        for r in done:
            t = int(r["tag"])
            assert int(r["d"]) == int(d_ref[t]), t
            assert np.array_equal(res[offs[t]:offs[t + 1]].numpy().view(np.uint32), bits_ref[t]), t
    finally:
        srv.stop()


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_every_form_matches_the_batch_path(pool, form):
    """Single, paired, and the two mixed in one burst (the per-request choice by load): bits, d_e and
    iteration counts equal the batch path's."""
    w, host, mask_base = pool
    n = w.n_tb
    words = [_tb_words(w, t) for t in range(n)]
    offs = np.concatenate([[0], np.cumsum(words)]).astype(np.int64)
    res = torch.zeros(int(offs[-1]), dtype=torch.int32).pin_memory()
    s = session_for(w, "i8")
    srv = Server(s, host, res, arena_bytes=1 << 26, max_inflight=256, paired=form[0], pair_threshold=form[1])
    try:
        recs = tb_records(w, mask_base, abi.SERVE_TB_NP, tags=np.arange(n), result_offsets=4 * offs[:-1])
        done = srv.replay(recs, np.zeros(n, np.int64), timeout_ms=20000)
        assert sorted(done["tag"].tolist()) == list(range(n))
        _check_forms(srv, form[2])
        st = srv.stats()
        assert st["requests"] == n and st["launches"] >= 1
        d_ref, bits_ref, it_ref = _batch_reference(w, range(n))
        for r in done:
            t = int(r["tag"])
            assert int(r["d"]) == int(d_ref[t]), t
            assert int(r["max_iters"]) == it_ref[t], t
            assert np.array_equal(res[offs[t]:offs[t + 1]].numpy().view(np.uint32), bits_ref[t]), t
    finally:
        srv.stop()


def test_form_flags_are_validated(pool):
    w, host, mask_base = pool
    with pytest.raises(ValueError):
        Server(session_for(w, "i8"), host, None, arena_bytes=1 << 24, max_inflight=8, paired="sometimes")
    with pytest.raises(LdpcError, match="EINVAL"):
        Server(session_for(w, "i8"), host, None, arena_bytes=1 << 24, max_inflight=8, pair_threshold=-1)


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_segmented_tbs_with_code_block_crcs_match_the_batch_path(form):
    """TBs whose code blocks carry their own CRC (payload n_cb (K - 24) - 24): the service infers that from
    payload_bits, stops blocks on a passing CRC and checks every CRC, like the batch path, bit for bit."""
    w = tb_pool(24, seed=17, max_cb=6, cb_crc=True)
    assert (w.cbs["flags"] == 1).any()
    raw, mask_base = pool_bytes(w)
    host = torch.from_numpy(raw).pin_memory()
    n = w.n_tb
    words = [_tb_words(w, t) for t in range(n)]
    offs = np.concatenate([[0], np.cumsum(words)]).astype(np.int64)
    res = torch.zeros(int(offs[-1]), dtype=torch.int32).pin_memory()
    s = session_for(w, "i8")
    plain = Server(session_for(w, "i8"), host, None, arena_bytes=1 << 24, max_inflight=8)
    try:
        seg = int(np.flatnonzero(w.tbs["n_cb"] > 1)[0])
        with pytest.raises(LdpcError, match="LDPC_SERVE_CB_CRC"):
            plain.submit(tb_records(w, mask_base, abi.SERVE_TB_NP, pool_index=[seg], tags=[0]))
    finally:
        plain.stop()
    srv = Server(s, host, res, arena_bytes=1 << 26, max_inflight=64, cb_crc=True, paired=form[0],
                 pair_threshold=form[1])
    try:
        recs = tb_records(w, mask_base, abi.SERVE_TB_NP, tags=np.arange(n), result_offsets=4 * offs[:-1])
        done = srv.replay(recs, np.zeros(n, np.int64), timeout_ms=20000)
        assert sorted(done["tag"].tolist()) == list(range(n))
        _check_forms(srv, form[2])
        d_ref, bits_ref, _ = _batch_reference(w, range(n))
        for r in done:
            t = int(r["tag"])
            assert int(r["d"]) == int(d_ref[t]), t
            assert np.array_equal(res[offs[t]:offs[t + 1]].numpy().view(np.uint32), bits_ref[t]), t
        assert 0 < int(done["d"].sum()) < n  # both outcomes occur at these SNRs
    finally:
        srv.stop()


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_redundancy_versions_through_the_service_match_the_batch_path(form):
    """Code blocks of redundancy versions 0-3 (k0 inside the circular buffer, wrapping it, repetition):
    the service's fused demap lands every bit on (k0 + e) mod Ncb and decodes the same columns as the
    batch path, bit for bit."""
    from workload.configs import cb_rv, redundancy_versions
    w = redundancy_versions(n_per=2, rates=(0.5, 0.3, 0.2), seed=15)
    assert sorted({cb_rv(c) for c in w.cbs}) == [0, 1, 2, 3]
    raw, mask_base = pool_bytes(w)
    host = torch.from_numpy(raw).pin_memory()
    n = w.n_tb
    words = [_tb_words(w, t) for t in range(n)]
    offs = np.concatenate([[0], np.cumsum(words)]).astype(np.int64)
    res = torch.zeros(int(offs[-1]), dtype=torch.int32).pin_memory()
    s = session_for(w, "i8")
    srv = Server(s, host, res, arena_bytes=1 << 24, max_inflight=64, paired=form[0], pair_threshold=form[1])
    try:
        recs = tb_records(w, mask_base, abi.SERVE_TB_NP, tags=np.arange(n), result_offsets=4 * offs[:-1])
        assert sorted(set(recs["rv"].tolist())) == [0, 1, 2, 3]
        bad = recs[:1].copy()
        bad["rv"] = 4
        with pytest.raises(LdpcError, match="rv"):
            srv.submit(bad)
        done = srv.replay(recs, np.zeros(n, np.int64), timeout_ms=20000)
        assert sorted(done["tag"].tolist()) == list(range(n))
        _check_forms(srv, form[2])
        d_ref, bits_ref, it_ref = _batch_reference(w, range(n))
        for r in done:
            t = int(r["tag"])
            assert int(r["d"]) == int(d_ref[t]), t
            assert int(r["max_iters"]) == it_ref[t], t
            assert np.array_equal(res[offs[t]:offs[t + 1]].numpy().view(np.uint32), bits_ref[t]), t
        assert 0 < int(done["d"].sum()) < n  # versions 1-2 at these rates are not all self-decodable
    finally:
        srv.stop()


@pytest.mark.parametrize("mode", ["f32", "i16"])
def test_float_and_int16_services_match_the_batch_path(mode):
    """The FP32 and INT16 serving loops (single form, messages in shared memory; shapes up to Z = 128 so
    that FP32 fits): bits, d_e and iteration counts equal the batch path in the same arithmetic; a shape
    whose FP32 state does not fit shared memory is refused."""
    w = tb_pool(24, seed=19, max_cb=5, zs=(32, 64, 128), snr_range_db=(3.0, 6.0))  # oracle: 3 of 24 pass
    raw, mask_base = pool_bytes(w)
    host = torch.from_numpy(raw).pin_memory()
    n = w.n_tb
    words = [_tb_words(w, t) for t in range(n)]
    offs = np.concatenate([[0], np.cumsum(words)]).astype(np.int64)
    res = torch.zeros(int(offs[-1]), dtype=torch.int32).pin_memory()
    s = session_for(w, mode)
    srv = Server(s, host, res, arena_bytes=1 << 26, max_inflight=64)
    try:
        recs = tb_records(w, mask_base, abi.SERVE_TB_NP, tags=np.arange(n), result_offsets=4 * offs[:-1])
        done = srv.replay(recs, np.zeros(n, np.int64), timeout_ms=20000)
        assert sorted(done["tag"].tolist()) == list(range(n))
        st = srv.stats()
        assert st["items_paired"] == 0 and st["items_single"] > 0
        d_ref, bits_ref, it_ref = _batch_reference(w, range(n), mode)
        for r in done:
            t = int(r["tag"])
            assert int(r["d"]) == int(d_ref[t]), t
            assert int(r["max_iters"]) == it_ref[t], t
            assert np.array_equal(res[offs[t]:offs[t + 1]].numpy().view(np.uint32), bits_ref[t]), t
        assert 0 < int(done["d"].sum()) < n
    finally:
        srv.stop()
    if mode == "f32":  # Z = 384 in FP32 (either base graph): too large for the loop's shared memory
        big = tb_pool(2, seed=3, max_cb=1, zs=(384,))
        raw2, mb2 = pool_bytes(big)
        host2 = torch.from_numpy(raw2).pin_memory()
        srv2 = Server(session_for(big, "f32"), host2, None, arena_bytes=1 << 24, max_inflight=8)
        try:
            with pytest.raises(LdpcError, match="shared memory"):
                srv2.submit(tb_records(big, mb2, abi.SERVE_TB_NP)[:1])
        finally:
            srv2.stop()


def test_two_loops_per_sm_is_withdrawn(pool):
    w, host, mask_base = pool
    with pytest.raises(LdpcError, match="withdrawn"):
        Server(session_for(w, "i8"), host, None, arena_bytes=1 << 24, max_inflight=8, loops_per_sm=2)
