"""Host side of the decode service's requests: the record layout the C-ABI expects (ldpc_serve_tb) and the
request builder's fields and pool layout (each TB's blocks' symbols and mask words back to back)."""
import numpy as np

from paper_2506_00167_gb300 import abi
from workload.configs import cb_rv, redundancy_versions
from workload.serving import pool_bytes, tb_pool, tb_records


def test_record_layout_matches_the_header():
    dt = abi.SERVE_TB_NP
    # int32 bg, Z, Qm, E, n_cb, n_sc, payload_bits; float inv_sigma2; int32 rv, pattern; int64 offsets;
    # u64 tag; int32 grid_sc, reserved
    want = [("bg", 0), ("Z", 4), ("Qm", 8), ("E", 12), ("n_cb", 16), ("n_sc", 20), ("payload_bits", 24),
            ("inv_sigma2", 28), ("rv", 32), ("pattern", 36), ("sym_offset", 40), ("mask_offset", 48),
            ("result_offset", 56), ("tag", 64), ("grid_sc", 72), ("reserved", 76)]
    assert [(n, dt.fields[n][1]) for n, _ in want] == want
    assert dt.itemsize == 80


def _check(w):
    raw, mask_base = pool_bytes(w)
    assert mask_base % 16 == 0
    recs = tb_records(w, mask_base, abi.SERVE_TB_NP, tags=np.arange(w.n_tb) + 100,
                      result_offsets=np.arange(w.n_tb) * 64)
    for t, r in enumerate(recs):
        tb = w.tbs[t]
        first, n = int(tb["first_cb"]), int(tb["n_cb"])
        c = w.cbs[first]
        for name in ("bg", "Z", "Qm", "E"):
            assert int(r[name]) == int(c[name]), (t, name)
            assert all(int(w.cbs[i][name]) == int(c[name]) for i in range(first, first + n))  # one shape per TB
        assert np.float32(r["inv_sigma2"]) == np.float32(c["inv_sigma2"])
        assert (int(r["n_cb"]), int(r["n_sc"]), int(r["payload_bits"])) == (n, int(tb["n_sc"]),
                                                                            int(tb["payload_bits"]))
        assert int(r["rv"]) == cb_rv(c) and int(r["pattern"]) == -1 and int(r["reserved"]) == 0
        assert (int(r["tag"]), int(r["result_offset"])) == (100 + t, 64 * t)
        # the blocks' symbols and mask words lie back to back where the record says
        n_re = int(c["E"]) // int(c["Qm"])
        mw = (n_re + 31) // 32
        so, mo = int(r["sym_offset"]), int(r["mask_offset"])
        assert so % 8 == 0 and mo % 4 == 0
        sym = raw[so:so + n * n_re * 8].view(np.complex64)
        msk = raw[mo:mo + n * mw * 4].view(np.uint32)
        for j in range(n):
            cj = w.cbs[first + j]
            ro, wo = int(cj["re_offset"]), int(cj["mask_word_offset"])
            assert np.array_equal(sym[j * n_re:(j + 1) * n_re], np.asarray(w.sym[ro:ro + n_re], np.complex64))
            assert np.array_equal(msk[j * mw:(j + 1) * mw], np.asarray(w.mask[wo:wo + mw], np.uint32))


def test_pool_requests_carry_their_blocks():
    _check(tb_pool(12, seed=21, max_cb=6, own_band_masks=True))


def test_redundancy_versions_reach_the_records():
    w = redundancy_versions(n_per=1, seed=15)
    _check(w)
    recs = tb_records(w, pool_bytes(w)[1], abi.SERVE_TB_NP)
    assert sorted(set(recs["rv"].tolist())) == [0, 1, 2, 3]
