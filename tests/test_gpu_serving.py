"""Continuous-batching decode service (GPU): the served stream (one URLLC codebook entry per slot on the slot's
shared grid, expanded on the device) against the batch path and the CPU oracle; same result alone and in the mix;
admission, idle relaunch, request validation."""
import time

import numpy as np
import pytest
import torch

from oracle import path as opath
from paper_2506_00167_gb300 import LdpcError, Server, abi
from workload.configs import subset
from workload.serving import CODEBOOK_PRB, codebook_bitmaps, pool_bytes, served_workload, slot_stream, tb_pool, \
    tb_records

from gpu_helpers import device_inputs, session_for

pytestmark = pytest.mark.gpu

# INT8 decode forms of the service: (paired, which item counters must be nonzero).  "auto" runs with a
# pair threshold equal to the first request's code blocks (see _thr): that request stays single (it never
# has more single-form items than blocks) and the burst behind it pairs once more items are in flight.
FORMS = [("auto", ("items_single", "items_paired")), (True, ("items_paired",)), (False, ("items_single",))]
FORM_IDS = ["auto", "paired", "single"]
BOOK = codebook_bitmaps()


def _thr(form, recs):
    return int(recs["n_cb"][0]) if form[0] == "auto" else 0


def _check_forms(srv, must):
    st = srv.stats()
    for k in ("items_single", "items_paired"):
        assert (st[k] > 0) == (k in must), st


class Stream:
    """A pool of unpunctured TBs and a served request stream over it: requests name their slot's codebook
    entry and their band's place on the slot's grid; ``sw`` is the same requests with the puncturing
    expanded on the host (the batch path's and the oracle's inputs), one TB per request."""

    def __init__(self, w, n_slots, n_ue, seed):
        self.w = w
        raw, self.mask_base = pool_bytes(w)
        self.host = torch.from_numpy(raw).pin_memory()
        self.s = slot_stream(n_slots, w.tbs["n_sc"], n_ue=n_ue, tb_per_slot=1.0, seed=seed)
        self.n = self.s["pool"].size
        self.sw = served_workload(w, self.s["pool"], self.s["pattern"], self.s["grid_sc"], BOOK)
        self.words = np.array([_tb_words(self.sw, t) for t in range(self.n)], np.int64)
        self.offs = np.concatenate([[0], np.cumsum(self.words)]).astype(np.int64)

    def records(self, idx=None, result_base=0):
        idx = np.arange(self.n) if idx is None else np.asarray(idx)
        return tb_records(self.w, self.mask_base, abi.SERVE_TB_NP, pool_index=self.s["pool"][idx], tags=idx,
                          result_offsets=4 * (result_base + self.offs[idx]), pattern=self.s["pattern"][idx],
                          grid_sc=self.s["grid_sc"][idx])

    def server(self, mode="i8", result_words=None, **kw):
        res = torch.zeros(int(self.offs[-1]) if result_words is None else result_words,
                          dtype=torch.int32).pin_memory()
        srv = Server(session_for(self.w, mode), self.host, res, codebook=(BOOK, CODEBOOK_PRB), **kw)
        return srv, res

    def bits(self, res, t, base=0):
        return res[base + self.offs[t]:base + self.offs[t + 1]].numpy().view(np.uint32)


@pytest.fixture(scope="module")
def stream():
    st = Stream(tb_pool(40, seed=7), n_slots=4, n_ue=12, seed=8)
    assert st.sw.mask.any()                       # URLLC punctured some of the requests
    return st


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
    the most iterations of any code block, per TB; and the demapped LLRs of each TB's blocks."""
    sub = subset(w, idx)
    s = session_for(sub, mode)
    b = s.batch(sub.cbs, sub.tbs, sub.slot_N)
    sym, mask = device_inputs(sub)
    out = s.run(b, sym, mask, b.alloc_outputs())
    torch.cuda.synchronize()
    bits = out["bits"].cpu().numpy().view(np.uint32)
    status = out["status"].cpu().numpy()
    llr = out["llr"].cpu().numpy()
    per_tb, iters, llrs = [], [], []
    for t in range(sub.n_tb):
        first, n = int(sub.tbs[t]["first_cb"]), int(sub.tbs[t]["n_cb"])
        c = sub.cbs[first]
        o = int(c["bits_word_offset"])
        per_tb.append(bits[o:o + _tb_words(sub, t)].copy())
        iters.append(int((status[first:first + n] & 0xFFFF).max()))
        l0 = int(c["llr_offset"])
        l1 = int(sub.cbs[first + n]["llr_offset"]) if first + n < sub.n_cb else llr.size
        llrs.append(llr[l0:l1].copy())
    return out["d"].cpu().numpy()[:sub.n_tb], per_tb, iters, llrs


def test_result_is_the_same_alone_and_in_the_mix(stream):
    st = stream
    n = st.n
    srv, res = st.server(result_words=2 * int(st.offs[-1]), arena_bytes=1 << 26, max_inflight=256)
    alone = [0, 3, 7, 11]
    # alone: one request at a time on an idle service
    d_alone = {}
    for t in alone:
        assert srv.submit(st.records([t])) == 1
        done = _wait(srv, 1)
        assert int(done["tag"][0]) == t
        d_alone[t] = int(done["d"][0])
    bits_alone = {t: st.bits(res, t).copy() for t in alone}
    # in the mix: every request of the stream arrives together (results into the second half of the pool)
    base = int(st.offs[-1])
    done = srv.replay(st.records(result_base=base), np.zeros(n, np.int64), timeout_ms=20000)
    assert sorted(done["tag"].tolist()) == list(range(n))
    d_mix = {int(r["tag"]): int(r["d"]) for r in done}
    for t in alone:
        assert d_mix[t] == d_alone[t]
        assert np.array_equal(st.bits(res, t, base), bits_alone[t])
    # and both equal the batch path on the host-expanded masks bit for bit, iteration counts included
    d_ref, bits_ref, it_ref, _ = _batch_reference(st.sw, range(n))
    it_mix = {int(r["tag"]): int(r["max_iters"]) for r in done}
    for t in range(n):
        assert d_mix[t] == int(d_ref[t]), t
        assert it_mix[t] == it_ref[t], t
        assert np.array_equal(st.bits(res, t, base), bits_ref[t]), t
    assert 0 < sum(d_mix.values()) < n
    lat = (done["t_complete_ns"] - done["t_submit_ns"]) / 1e3
    assert np.all(lat > 0)
    srv.stop()


def test_device_expansion_equals_host_mask_words(stream):
    """The same requests once as (codebook entry, grid offset) and once as explicit mask words (the host
    expansion laid into a second pool): identical bits, d_e and iterations."""
    st = stream
    n = st.n
    sw = st.sw
    raw2, mb2 = pool_bytes(sw)
    host2 = torch.from_numpy(raw2).pin_memory()
    res2 = torch.zeros(int(st.offs[-1]), dtype=torch.int32).pin_memory()
    srv2 = Server(session_for(sw, "i8"), host2, res2, arena_bytes=1 << 26, max_inflight=256)
    srv, res = st.server(arena_bytes=1 << 26, max_inflight=256)
    try:
        recs2 = tb_records(sw, mb2, abi.SERVE_TB_NP, tags=np.arange(n), result_offsets=4 * st.offs[:-1])
        assert np.all(recs2["pattern"] == -1)
        d2 = srv2.replay(recs2, np.zeros(n, np.int64), timeout_ms=20000)
        d1 = srv.replay(st.records(), np.zeros(n, np.int64), timeout_ms=20000)
        a = {int(r["tag"]): (int(r["d"]), int(r["max_iters"])) for r in d1}
        b = {int(r["tag"]): (int(r["d"]), int(r["max_iters"])) for r in d2}
        assert a == b
        assert np.array_equal(res.numpy(), res2.numpy())
    finally:
        srv.stop()
        srv2.stop()


def _oracle_parity(st, mode, srv_kw):
    """Service vs the CPU oracle on the same requests (the oracle demaps and decodes on its own: float64
    demap, then the mode's arithmetic).  Where the GPU's demapped LLRs of a TB equal the oracle's (integer
    modes: all but the rare LLR on a rounding boundary), bits, d_e and iterations must be identical; TB
    outcomes agree on all but 1 % (at least 1) of the TBs; a TB whose CRC passes carries exactly the
    information bits that were sent."""
    n = st.n
    srv, res = st.server(mode, arena_bytes=1 << 26, max_inflight=256, **srv_kw)
    try:
        done = srv.replay(st.records(), np.zeros(n, np.int64), timeout_ms=30000)
    finally:
        srv.stop()
    got = {int(r["tag"]): r for r in done}
    ref = opath.run(st.sw, mode, 10, True)
    _, _, _, llr_gpu = _batch_reference(st.sw, range(n), mode)
    same_llr = disagree = 0
    for t in range(n):
        tb = st.sw.tbs[t]
        first, ncb = int(tb["first_cb"]), int(tb["n_cb"])
        c = st.sw.cbs[first]
        l0 = int(c["llr_offset"])
        l1 = int(st.sw.cbs[first + ncb]["llr_offset"]) if first + ncb < st.sw.n_cb else ref["llr"].size
        o = int(c["bits_word_offset"])
        want_bits = ref["words"][o:o + _tb_words(st.sw, t)]
        want_it = int((ref["status"][first:first + ncb] & 0xFFFF).max())
        if np.array_equal(llr_gpu[t], ref["llr"][l0:l1]):
            same_llr += 1
            assert int(got[t]["d"]) == int(ref["d"][t]), t
            assert int(got[t]["max_iters"]) == want_it, t
            assert np.array_equal(st.bits(res, t), want_bits), t
        disagree += int(got[t]["d"]) != int(ref["d"][t])
        if int(got[t]["d"]):
            assert np.array_equal(st.bits(res, t), st.sw.info_words[o:o + _tb_words(st.sw, t)]), t
    if mode != "f32":  # float32 demaps differ from float64 ones in the last bits, so only integers match whole
        assert same_llr >= n // 2, (same_llr, n)
    assert disagree <= max(1, n // 100), disagree
    return got, ref


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_int8_service_matches_the_oracle(stream, form):
    got, ref = _oracle_parity(stream, "i8", dict(paired=form[0], pair_threshold=_thr(form, stream.records())))
    assert 0 < int(ref["d"].sum()) < stream.n


@pytest.fixture(scope="module")
def small_stream():
    """Shapes up to Z = 128 (messages in shared memory for INT16; FP32's are in device memory)."""
    return Stream(tb_pool(24, seed=19, max_cb=5, zs=(32, 64, 128)), n_slots=3, n_ue=10, seed=10)


@pytest.mark.parametrize("mode", ["f32", "i16"])
def test_float_and_int16_services_match_the_oracle(small_stream, mode):
    got, ref = _oracle_parity(small_stream, mode, {})
    assert 0 < int(ref["d"].sum()) < small_stream.n


def test_fp32_service_on_the_full_stream_matches_the_oracle(stream):
    """FP32 on the served stream's shapes up to Z = 384 (its check messages in a device-memory slot per
    loop group)."""
    got, ref = _oracle_parity(stream, "f32", {})
    assert 0 < int(ref["d"].sum()) < stream.n


def test_admission_waits_for_memory(stream):
    st = stream
    need = [_tb_words(st.sw, t) + int(st.sw.tbs[t]["n_cb"]) for t in range(3)]
    srv, _ = st.server(arena_bytes=4 * (need[0] + need[1]), max_inflight=64)
    recs = st.records([0, 1, 2])
    assert srv.submit(recs) == 2          # the third does not fit the arena yet
    done = _wait(srv, 2)
    assert sorted(done["tag"].tolist()) == [0, 1]
    assert srv.submit(recs[2:]) == 1      # admitted once the first two freed their space
    assert _wait(srv, 1)["tag"][0] == 2
    srv.stop()


def test_idle_loop_is_relaunched_and_bad_requests_rejected(stream):
    st = stream
    srv, _ = st.server(arena_bytes=1 << 24, max_inflight=16, idle_timeout_us=2000)
    rec = st.records([5])
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
    bad["sym_offset"] = st.host.numel()
    with pytest.raises(LdpcError, match="host pool"):
        srv.submit(bad)
    bad = rec.copy()
    bad["pattern"] = BOOK.shape[0]        # not in the codebook
    with pytest.raises(LdpcError, match="codebook"):
        srv.submit(bad)
    bad = rec.copy()
    bad["n_sc"] = 12                      # the TB does not fit a 12-subcarrier band in one slot
    with pytest.raises(LdpcError, match="band"):
        srv.submit(bad)
    bad = rec.copy()
    bad["reserved"] = 1
    with pytest.raises(LdpcError, match="reserved"):
        srv.submit(bad)
    srv.stop()
    # a service started without a codebook refuses requests that name an entry
    plain = Server(session_for(st.w, "i8"), st.host, None, arena_bytes=1 << 24, max_inflight=8)
    try:
        with pytest.raises(LdpcError, match="codebook"):
            plain.submit(rec)
    finally:
        plain.stop()


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
    recs = tb_records(w, mask_base, abi.SERVE_TB_NP, tags=np.arange(n), result_offsets=4 * offs[:-1])
    srv = Server(s, host, res, arena_bytes=1 << 24, max_inflight=64, paired=form[0], pair_threshold=_thr(form, recs))
    try:
        done = srv.replay(recs, np.zeros(n, np.int64), timeout_ms=20000)
        assert sorted(done["tag"].tolist()) == list(range(n))
        _check_forms(srv, form[1])
        d_ref, bits_ref, _, _ = _batch_reference(w, range(n))
        for r in done:
            t = int(r["tag"])
            assert int(r["d"]) == int(d_ref[t]), t
            assert np.array_equal(res[offs[t]:offs[t + 1]].numpy().view(np.uint32), bits_ref[t]), t
    finally:
        srv.stop()


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_every_form_matches_the_batch_path(stream, form):
    """Single, paired, and the two mixed in one burst (the per-request choice by load): bits, d_e and
    iteration counts equal the batch path's on every request."""
    st = stream
    n = st.n
    srv, res = st.server(arena_bytes=1 << 26, max_inflight=256, paired=form[0],
                         pair_threshold=_thr(form, st.records()))
    try:
        done = srv.replay(st.records(), np.zeros(n, np.int64), timeout_ms=20000)
        assert sorted(done["tag"].tolist()) == list(range(n))
        _check_forms(srv, form[1])
        stats = srv.stats()
        assert stats["requests"] == n and stats["launches"] >= 1
        d_ref, bits_ref, it_ref, _ = _batch_reference(st.sw, range(n))
        for r in done:
            t = int(r["tag"])
            assert int(r["d"]) == int(d_ref[t]), t
            assert int(r["max_iters"]) == it_ref[t], t
            assert np.array_equal(st.bits(res, t), bits_ref[t]), t
    finally:
        srv.stop()


def test_form_flags_are_validated(stream):
    w, host = stream.w, stream.host
    with pytest.raises(ValueError):
        Server(session_for(w, "i8"), host, None, arena_bytes=1 << 24, max_inflight=8, paired="sometimes")
    with pytest.raises(LdpcError, match="EINVAL"):
        Server(session_for(w, "i8"), host, None, arena_bytes=1 << 24, max_inflight=8, pair_threshold=-1)
    with pytest.raises(ValueError):
        Server(session_for(w, "i8"), host, None, arena_bytes=1 << 24, max_inflight=8,
               codebook=(BOOK[:, :6], CODEBOOK_PRB))


@pytest.fixture(scope="module")
def seg_stream():
    st = Stream(tb_pool(24, seed=17, max_cb=6, cb_crc=True), n_slots=3, n_ue=10, seed=9)
    assert (st.w.cbs["flags"] == 1).any()
    return st


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_segmented_tbs_with_code_block_crcs_match_the_batch_path(seg_stream, form):
    """TBs whose code blocks carry their own CRC (payload n_cb (K - 24) - 24): the service infers that from
    payload_bits, stops blocks on a passing CRC and checks every CRC, like the batch path, bit for bit."""
    st = seg_stream
    n = st.n
    plain = Server(session_for(st.w, "i8"), st.host, None, arena_bytes=1 << 24, max_inflight=8,
                   codebook=(BOOK, CODEBOOK_PRB))
    try:
        seg = int(np.flatnonzero(st.sw.tbs["n_cb"] > 1)[0])
        with pytest.raises(LdpcError, match="LDPC_SERVE_CB_CRC"):
            plain.submit(st.records([seg]))
    finally:
        plain.stop()
    srv, res = st.server(arena_bytes=1 << 26, max_inflight=64, cb_crc=True, paired=form[0],
                         pair_threshold=_thr(form, st.records()))
    try:
        done = srv.replay(st.records(), np.zeros(n, np.int64), timeout_ms=20000)
        assert sorted(done["tag"].tolist()) == list(range(n))
        _check_forms(srv, form[1])
        d_ref, bits_ref, _, _ = _batch_reference(st.sw, range(n))
        for r in done:
            t = int(r["tag"])
            assert int(r["d"]) == int(d_ref[t]), t
            assert np.array_equal(st.bits(res, t), bits_ref[t]), t
        assert 0 < int(done["d"].sum()) < n  # both outcomes occur (oracle: 15 of 36 pass)
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
    recs = tb_records(w, mask_base, abi.SERVE_TB_NP, tags=np.arange(n), result_offsets=4 * offs[:-1])
    srv = Server(s, host, res, arena_bytes=1 << 24, max_inflight=64, paired=form[0], pair_threshold=_thr(form, recs))
    try:
        assert sorted(set(recs["rv"].tolist())) == [0, 1, 2, 3]
        bad = recs[:1].copy()
        bad["rv"] = 4
        with pytest.raises(LdpcError, match="rv"):
            srv.submit(bad)
        done = srv.replay(recs, np.zeros(n, np.int64), timeout_ms=20000)
        assert sorted(done["tag"].tolist()) == list(range(n))
        _check_forms(srv, form[1])
        d_ref, bits_ref, it_ref, _ = _batch_reference(w, range(n))
        for r in done:
            t = int(r["tag"])
            assert int(r["d"]) == int(d_ref[t]), t
            assert int(r["max_iters"]) == it_ref[t], t
            assert np.array_equal(res[offs[t]:offs[t + 1]].numpy().view(np.uint32), bits_ref[t]), t
        assert 0 < int(done["d"].sum()) < n  # versions 1-2 at these rates are not all self-decodable
    finally:
        srv.stop()


@pytest.mark.parametrize("mode", ["f32", "i16"])
def test_float_and_int16_services_match_the_batch_path(small_stream, mode):
    """The FP32 and INT16 serving loops (single form): bits, d_e and iteration counts equal the batch path
    in the same arithmetic, on shapes up to Z = 128 and, in FP32, on Z = 384 shapes too."""
    st = small_stream
    n = st.n
    srv, res = st.server(mode, arena_bytes=1 << 26, max_inflight=64)
    try:
        done = srv.replay(st.records(), np.zeros(n, np.int64), timeout_ms=20000)
        assert sorted(done["tag"].tolist()) == list(range(n))
        stats = srv.stats()
        assert stats["items_paired"] == 0 and stats["items_single"] > 0
        d_ref, bits_ref, it_ref, _ = _batch_reference(st.sw, range(n), mode)
        for r in done:
            t = int(r["tag"])
            assert int(r["d"]) == int(d_ref[t]), t
            assert int(r["max_iters"]) == it_ref[t], t
            assert np.array_equal(st.bits(res, t), bits_ref[t]), t
        assert 0 < int(done["d"].sum()) < n
    finally:
        srv.stop()
    if mode == "f32":  # Z = 384 in FP32 (either base graph): the messages in device memory
        big = Stream(tb_pool(6, seed=3, max_cb=2, zs=(384,)), n_slots=2, n_ue=4, seed=11)
        srv2, res2 = big.server("f32", arena_bytes=1 << 26, max_inflight=16)
        try:
            done = srv2.replay(big.records(), np.zeros(big.n, np.int64), timeout_ms=20000)
            assert sorted(done["tag"].tolist()) == list(range(big.n))
            d_ref, bits_ref, it_ref, _ = _batch_reference(big.sw, range(big.n), "f32")
            for r in done:
                t = int(r["tag"])
                assert int(r["d"]) == int(d_ref[t]), t
                assert int(r["max_iters"]) == it_ref[t], t
                assert np.array_equal(big.bits(res2, t), bits_ref[t]), t
        finally:
            srv2.stop()


def test_two_loops_per_sm_is_withdrawn(stream):
    with pytest.raises(LdpcError, match="withdrawn"):
        Server(session_for(stream.w, "i8"), stream.host, None, arena_bytes=1 << 24, max_inflight=8, loops_per_sm=2)
