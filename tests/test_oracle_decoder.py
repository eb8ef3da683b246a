"""Pins for the oracle's layered offset-min-sum decoder."""
import itertools

import numpy as np
import pytest

from oracle import decoder, demap, encoder, path
from workload import large_fp32, tiny_fp32, mixed
from workload.basegraph import make_base_graph, tree_base_graph


def _brute_force_maxlog(bg, Z, lam):
    """L_v = min_{c in C, c_v=1} sum_u c_u lam_u - min_{c in C, c_v=0} sum_u c_u lam_u, by enumeration."""
    n = bg.nb * Z
    words = np.array(list(itertools.product((0, 1), repeat=n)), dtype=np.uint8)
    ok = np.array([not encoder.syndrome(bg, Z, w).any() for w in words])
    C = words[ok]
    cost = C.astype(lam.dtype) @ lam if lam.dtype.kind == "f" else C.astype(np.int64) @ lam
    out = np.empty(n, dtype=cost.dtype)
    for v in range(n):
        out[v] = cost[C[:, v] == 1].min() - cost[C[:, v] == 0].min()
    return out, C


def test_tree_code_minsum_equals_bruteforce_maxlog_float():
    bg = tree_base_graph()
    Z = 2
    rng = np.random.default_rng(11)
    for trial in range(4):
        lam = rng.normal(0.0, 2.0, size=bg.nb * Z)
        ml, C = _brute_force_maxlog(bg, Z, lam)
        assert C.shape[0] == 2 ** (bg.nb * Z - bg.mb * Z)  # forest: all 6 checks independent
        _, _, _, L = decoder.layered_oms(lam[None], bg, Z, bg.mb, 12, False,
                                         decoder.FloatArith(0.0), return_L=True)
        assert np.allclose(L[0], ml, atol=1e-12, rtol=0)


def test_tree_code_minsum_equals_bruteforce_maxlog_integer():
    bg = tree_base_graph()
    Z = 2
    rng = np.random.default_rng(12)
    exact = decoder.IntArith(beta=0, msg_sat=10 ** 9, post_sat=10 ** 12)
    for trial in range(4):
        lam = rng.integers(-40, 41, size=bg.nb * Z).astype(np.int64)
        ml, _ = _brute_force_maxlog(bg, Z, lam)
        _, _, _, L = decoder.layered_oms(lam[None], bg, Z, bg.mb, 12, False, exact, return_L=True)
        assert np.array_equal(L[0], ml)


def test_offset_changes_tree_result():
    # a plausible slip (offset never applied) would pass the beta=0 test; this
    # one fixes the beta=0.5 value on a two-check path by hand.
    bg = tree_base_graph()
    Z = 2
    lam = np.zeros(bg.nb * Z)
    # variables in column 4 (row 1 only) get the extrinsic of row 1 from cols 3 and 5
    lam[3 * Z:4 * Z] = 3.0
    lam[5 * Z:6 * Z] = 2.0
    _, _, _, L = decoder.layered_oms(lam[None], bg, Z, bg.mb, 1, False, decoder.FloatArith(0.5),
                                     return_L=True)
    # first iteration, row 0 runs first: column 3 has three erased neighbours -> R = 0.
    # row 1 for column 4: Q3 = 3, Q5 = 2 (row 2 not yet run) -> R = min(3,2) - 0.5 = 1.5
    assert np.allclose(L[0, 4 * Z:5 * Z], 1.5)


def test_all_zero_llr_decodes_to_zero_word():
    bg = make_base_graph("bg1")
    Z = 16
    m = bg.m_eff(Z, 22 * Z * 2)
    llr = np.zeros((2, (bg.kb + m) * Z))
    bits, iters, ok = decoder.layered_oms(llr, bg, Z, m, 10, True)
    assert not bits.any() and np.all(iters == 1) and np.all(ok)
    bits, iters, ok = decoder.layered_oms(llr.astype(np.int64), bg, Z, m, 10, True, decoder.INT8)
    assert not bits.any() and np.all(iters == 1) and np.all(ok)


@pytest.mark.parametrize("mode", ["f64", "i8", "i16"])
def test_noiseless_decodes_exactly(mode):
    w = large_fp32(n_cw=6, noiseless=True, with_urllc=False)
    out = path.run(w, mode, max_iter=10, early_term=True)
    assert not path.block_errors(w, out["words"]).any()
    st = out["status"]
    assert np.all(st >> 16 == 1)
    assert np.all((st & 0xFFFF) <= 2)
    assert np.all(out["d"] == 1)
    assert np.all(out["reward"] == 0.0)


def test_noiseless_with_urllc_puncturing_decodes():
    w = large_fp32(n_cw=6, noiseless=True, with_urllc=True, seed=5)
    out = path.run(w, "f64", max_iter=10, early_term=True)
    assert not path.block_errors(w, out["words"]).any()


def test_tiny_code_noiseless_no_et_runs_all_iterations():
    w = tiny_fp32(n_per_point=4, ebn0_points=(3,), noiseless=True)
    out = path.run(w, "f64", max_iter=8, early_term=False)
    assert not path.block_errors(w, out["words"]).any()
    assert np.all(out["status"] & 0xFFFF == 8)


def test_all_zero_codeword_high_snr():
    bg = make_base_graph("bg2")
    Z, Qm, E = 32, 4, 640
    rng = np.random.default_rng(4)
    pts, labels = demap.constellation(Qm)
    x = np.full(E // Qm, pts[0])
    y = x + np.sqrt(0.01 / 2) * (rng.standard_normal(x.size) + 1j * rng.standard_normal(x.size))
    llr = demap.demap_cb(y, np.zeros(x.size, bool), bg, Z, Qm, E, 100.0)
    _, m_eff, _ = demap.bg_geometry(bg, Z, E)
    bits, iters, ok = decoder.layered_oms(llr[None], bg, Z, m_eff, 10, True)
    assert not bits.any() and ok[0]


@pytest.mark.parametrize("arith", [decoder.F64, decoder.INT8])
def test_dropped_rows_are_exact(arith):
    # rows >= m_eff hang on never-sent degree-1 parity columns: decoding on all
    # mb rows (extra LLRs 0) leaves the first n_eff columns bit-identical.
    w = large_fp32(n_cw=2, snr_points=(8,))
    bg = w.bgs[0]
    Z, E = 384, 16896
    t0, m_eff, n_eff = demap.bg_geometry(bg, Z, E)
    llr = demap.demap_workload(w)[:n_eff * Z]
    if isinstance(arith, decoder.IntArith):
        llr = demap.quantise(llr, 4.0, 63)
    full = np.zeros(bg.nb * Z, dtype=llr.dtype)
    full[:n_eff * Z] = llr
    _, _, _, L1 = decoder.layered_oms(llr[None], bg, Z, m_eff, 3, False, arith, return_L=True)
    _, _, _, L2 = decoder.layered_oms(full[None], bg, Z, bg.mb, 3, False, arith, return_L=True)
    assert np.array_equal(L1[0], L2[0, :n_eff * Z])


def test_syndrome_ok_means_codeword():
    w = mixed(n_slots=2, ues_per_slot=3, max_cb=2)
    llr = demap.demap_workload(w)
    words, status, L = decoder.decode_workload(w, llr, 10, True, return_L=True)
    n_ok = 0
    for i in range(w.n_cb):
        bg, Z, t0, m_eff, n_eff = w.cb_geometry(i)
        lo = int(w.cbs[i]["llr_offset"])
        hard = np.zeros(bg.nb * Z, np.uint8)
        hard[:n_eff * Z] = L[lo:lo + n_eff * Z] < 0
        s = encoder.syndrome(bg, Z, hard, rows=range(m_eff))
        assert (not s.any()) == bool(status[i] >> 16)
        n_ok += int(status[i] >> 16)
    assert n_ok > 0


def test_int8_state_stays_saturated_and_deterministic():
    w = large_fp32(n_cw=3, snr_points=(7,))
    llr = demap.quantise(demap.demap_workload(w), 4.0, 63)
    a = decoder.decode_workload(w, llr, 10, True, decoder.INT8, return_L=True)
    b = decoder.decode_workload(w, llr, 10, True, decoder.INT8, return_L=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.abs(a[2]).max() <= 127


def test_float32_run_close_to_float64():
    w = large_fp32(n_cw=8, snr_points=(9,))
    llr = demap.demap_workload(w)
    w64, s64 = decoder.decode_workload(w, llr, 10, True, decoder.F64)
    w32, s32 = decoder.decode_workload(w, llr.astype(np.float32), 10, True, decoder.F32)
    assert np.array_equal(w64, w32)


def _star3():
    """Three degree-2 checks sharing variable 0: rows {0,1}, {0,2}, {0,3}; Z = 1 (every shift 0)."""
    from workload.basegraph import custom_base_graph
    return custom_base_graph("star3", 3, 4, 1, 3, 0, {(0, 0): 0, (0, 1): 0, (1, 0): 0, (1, 2): 0,
                                                       (2, 0): 0, (2, 3): 0})


def _final_L(arith, llr, iters):
    _, _, _, L = decoder.layered_oms(np.array([llr], dtype=np.int64), _star3(), 1, 3, iters, False, arith,
                                     return_L=True)
    return L[0].tolist()


def test_int8_saturation_worked_by_hand():
    """INT8 rule (precision configuration: 6-bit saturated magnitude, offset 1 LSB): Q = sat127(L - R),
    |Q| clamped to 63 for the minima, R' = sgn * max(m - 1, 0), L = sat127(Q + R').  Channel [10, -30, 63, 63].

    Iteration 1 (R = 0):
      row {0,1}: Q = [10, -30]; |Q| = [10, 30]; m1 = 10 (edge 0), m2 = 30; one negative -> parity 1.
                 R' = [-(30-1), +(10-1)] = [-29, 9];  L0 = 10 - 29 = -19, L1 = -30 + 9 = -21.
      row {0,2}: Q = [-19, 63]; m1 = 19 (edge 0), m2 = 63; parity 1.  R' = [+62, -18]; L0 = 43, L2 = 45.
      row {0,3}: Q = [43, 63]; m1 = 43, m2 = 63; parity 0.  R' = [62, 42]; L0 = 105, L3 = 105.
      -> L = [105, -21, 45, 105].
    Iteration 2:
      row {0,1} (R = [-29, 9]): Q = [sat127(105 + 29), -21 - 9] = [127, -30]   <- Q saturates
                 |Q| clamped: [63, 30] -> m1 = 30 (edge 1), m2 = 63; parity 1.
                 R' = [-(30-1), +(63-1)] = [-29, 62]   <- the clamped |Q| feeds edge 1's message
                 L0 = 127 - 29 = 98, L1 = -30 + 62 = 32.
      row {0,2} (R = [62, -18]): Q = [98 - 62, 45 + 18] = [36, 63]; m1 = 36, m2 = 63; parity 0.
                 R' = [62, 35]; L0 = 98, L2 = 98.
      row {0,3} (R = [62, 42]): Q = [36, 63]; R' = [62, 35]; L0 = 98, L3 = 98.
      -> L = [98, 32, 98, 98].
    Plausible slips and what they would give: no Q saturation -> L0 = 105 after iteration 2; Q saturated
    at 63 -> L0 = 34; |Q| not clamped -> R'_1 = 126, L1 = 96; the message R' clamped to 63 instead of |Q|
    -> L1 = 33; L saturated at 63 -> L0 = 63 after iteration 1.  (Clamping |Q| before or after taking
    the minima gives the same messages: the clamp is monotone, so it commutes with min and second min.)
    """
    assert _final_L(decoder.INT8, [10, -30, 63, 63], 1) == [105, -21, 45, 105]
    assert _final_L(decoder.INT8, [10, -30, 63, 63], 2) == [98, 32, 98, 98]


def test_int16_saturation_worked_by_hand():
    """INT16 rule: Q and L saturate at +-32767, |Q| clamped to 1023, offset 1.  Channel [32000, -500, 2000,
    2000] (large inputs reach the posterior limit within two iterations).

    Iteration 1:
      row {0,1}: Q = [32000, -500]; |Q| = [1023, 500] -> m1 = 500 (edge 1), m2 = 1023; parity 1.
                 R' = [-(500-1), +(1023-1)] = [-499, 1022]; L0 = 31501, L1 = 522.
      row {0,2}: Q = [31501, 2000]; |Q| = [1023, 1023] -> m1 = m2 = 1023; parity 0.  R' = [1022, 1022];
                 L0 = 32523, L2 = 3022.
      row {0,3}: Q = [32523, 2000]; R' = [1022, 1022]; L0 = sat(33545) = 32767   <- L saturates
                 L3 = 3022.   -> L = [32767, 522, 3022, 3022].
    Iteration 2:
      row {0,1} (R = [-499, 1022]): Q = [sat(32767 + 499), 522 - 1022] = [32767, -500]   <- Q saturates
                 R' = [-499, 1022]; L0 = 32268, L1 = 522.
      row {0,2} (R = [1022, 1022]): Q = [31246, 2000]; R' = [1022, 1022]; L0 = 32268, L2 = 3022.
      row {0,3}: the same; L3 = 3022.   -> L = [32268, 522, 3022, 3022].
    Slips: no Q saturation -> L0 = 32767 after iteration 2; |Q| not clamped -> R'_1 = 31999 in iteration 1;
    the INT8 limits -> every value differs.
    """
    assert _final_L(decoder.INT16, [32000, -500, 2000, 2000], 1) == [32767, 522, 3022, 3022]
    assert _final_L(decoder.INT16, [32000, -500, 2000, 2000], 2) == [32268, 522, 3022, 3022]
