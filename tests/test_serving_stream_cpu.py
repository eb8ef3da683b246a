"""The served request stream's URLLC puncturing (Sec. III-A mini-slot preemption; one codebook entry per slot on
the slot's shared subcarrier grid): the stream's structure, and the host expansion of (entry, band offset) into
mask words against the workload builder's own resource-element mapping of a whole slot."""
import numpy as np

from workload.configs import N_MINISLOT, N_SYM, TBSpec, build, default_bgs
from workload.serving import (CODEBOOK_PRB, Q_MINISLOT, codebook, codebook_bitmaps, expand_mask, served_workload,
                              slot_stream, tb_pool)


def test_codebook_bitmaps_hold_the_runs():
    book = codebook()
    bm = codebook_bitmaps()
    assert bm.shape == (128, N_MINISLOT, -(-CODEBOOK_PRB // 32))
    for cid, (mask, runs) in enumerate(book):
        assert mask == cid
        want = np.zeros((N_MINISLOT, CODEBOOK_PRB), bool)
        for m, st, ln in runs:
            assert 4 <= ln <= 12 and 0 <= st and st + ln <= CODEBOOK_PRB
            want[m, st:st + ln] = True
        assert sorted(m for m, _, _ in runs) == [m for m in range(N_MINISLOT) if (cid >> m) & 1]
        got = np.unpackbits(bm[cid].view(np.uint8), axis=1, bitorder="little")[:, :CODEBOOK_PRB].astype(bool)
        assert np.array_equal(got, want), cid


def test_one_entry_per_slot_and_bands_side_by_side():
    n_sc = np.array([24, 36, 120, 12, 600], np.int64)
    s = slot_stream(3000, n_sc, n_ue=40, tb_per_slot=1.0, seed=9)
    assert np.all(np.diff(s["t_ns"]) >= 0) and np.all(s["t_ns"] == s["slot"] * 125_000)
    for slot in range(0, 3000, 97):
        sel = np.flatnonzero(s["slot"] == slot)
        if sel.size == 0:
            continue
        assert np.unique(s["pattern"][sel]).size == 1      # one codebook entry per slot
        w = n_sc[s["pool"][sel]]
        assert np.array_equal(s["grid_sc"][sel], np.concatenate([[0], np.cumsum(w)[:-1]]))  # contiguous bands
    # mini-slot bits i.i.d. with q = 1 - 0.92^12 over the slots
    pat = np.array([s["pattern"][np.flatnonzero(s["slot"] == k)[0]] for k in range(3000)
                    if np.any(s["slot"] == k)])
    frac = ((pat[:, None] >> np.arange(N_MINISLOT)) & 1).mean(axis=0)
    sd = np.sqrt(Q_MINISLOT * (1 - Q_MINISLOT) / pat.size)
    assert np.all(np.abs(frac - Q_MINISLOT) < 5 * sd), frac


def test_expansion_matches_the_builders_slot_mapping():
    """Requests of one slot expanded one by one equal the builder's masks for the same TBs laid out as one slot
    (users side by side from subcarrier 0) under the entry's runs repeated every CODEBOOK_PRB PRBs."""
    pool = tb_pool(6, seed=31, max_cb=4, zs=(32, 64))
    bm = codebook_bitmaps()
    book = codebook()
    idx = [3, 0, 5, 5, 1]
    width = [int(pool.tbs[t]["n_sc"]) for t in idx]
    grid = np.concatenate([[0], np.cumsum(width)[:-1]])
    bgs = default_bgs()
    for cid in (0b1010101, 127, 6):
        total = int(np.sum(width))
        P = np.zeros((N_SYM, total), bool)
        for m, st, ln in book[cid][1]:
            for rep in range(0, total // 12 + CODEBOOK_PRB, CODEBOOK_PRB):
                a, b = 12 * (rep + st), 12 * (rep + st + ln)
                P[2 * m:2 * m + 2, a:min(b, total)] = True
        specs = []
        for t, g in zip(idx, grid):
            c = pool.cbs[int(pool.tbs[t]["first_cb"])]
            specs.append(TBSpec(0, int(c["bg"]), int(c["Z"]), int(c["Qm"]), int(c["E"]), int(pool.tbs[t]["n_cb"]),
                                1.0, int(g), int(pool.tbs[t]["n_sc"])))
        ref = build("slot", bgs, specs, [total], [P], seed=1, noiseless=True)
        sw = served_workload(pool, idx, [cid] * len(idx), grid, bm)
        assert np.array_equal(sw.mask, ref.mask), cid
        got = np.concatenate([np.concatenate(expand_mask(pool, t, cid, int(g), bm)) for t, g in zip(idx, grid)])
        assert np.array_equal(got, ref.mask)
    # a slot with no URLLC arrival punctures nothing
    assert not np.any(served_workload(pool, idx, [0] * len(idx), grid, bm).mask)
