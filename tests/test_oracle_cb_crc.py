"""Pins for the per-code-block CRC of segmented transport blocks: the CRC-24B generator, the
segmentation, the TB check over the segments, and CRC-aided early termination in the oracle decoder."""
import os

import numpy as np
import pytest

from oracle import crc, decoder, demap, goodput
from workload import tx
from workload.configs import segmented

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
POLYS = [crc.POLY, crc.POLY_B]


def _catalogue():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "crc24_check_values.txt"))
            if ln.strip() and not ln.startswith("#")]
    return [(int(a, 16), int(b, 16)) for a, b in rows]


def test_check_values_match_the_public_catalogue():
    msg = np.frombuffer(b"123456789", dtype=np.uint8)
    bits = ((msg[:, None] >> np.arange(7, -1, -1)[None, :]) & 1).reshape(1, -1)
    table = _catalogue()
    assert {p for p, _ in table} == set(POLYS)
    for poly, check in table:
        assert crc.remainder_bitwise(bits, poly)[0] == check
        assert crc.remainder_table(bits, poly)[0] == check


@pytest.mark.parametrize("poly", POLYS)
def test_codeword_generator_and_single_terms(poly):
    rng = np.random.default_rng(21)
    msg = rng.integers(0, 2, size=(12, 160), dtype=np.uint8)
    word = np.concatenate([msg, crc.crc_bits(msg, poly)], axis=1)
    assert np.all(crc.remainder_bitwise(word, poly) == 0)
    g = (1 << 24) | poly
    gb = np.array([(g >> (24 - i)) & 1 for i in range(25)], dtype=np.uint8)
    assert crc.remainder_bitwise(gb, poly)[0] == 0
    for k in range(24):
        e = np.zeros(24, np.uint8)
        e[23 - k] = 1
        assert crc.remainder_bitwise(e, poly)[0] != 0


def test_crc24b_detects_every_burst_up_to_24():
    rng = np.random.default_rng(22)
    msg = rng.integers(0, 2, size=(1, 48), dtype=np.uint8)
    word = np.concatenate([msg, crc.crc_bits(msg, crc.POLY_B)], axis=1)[0]
    n = word.size
    errs = []
    for length in range(1, 25):
        for start in range(0, n - length + 1):
            e = np.zeros(n, np.uint8)
            e[start] = 1
            e[start + length - 1] = 1
            if length > 2:
                e[start + 1:start + length - 1] = rng.integers(0, 2, size=length - 2)
            errs.append(word ^ e)
    assert np.all(crc.remainder_bitwise(np.array(errs), crc.POLY_B) != 0)


def test_crc24b_bitwise_matches_table_and_transmitter():
    rng = np.random.default_rng(23)
    m = rng.integers(0, 2, size=(10, 8 * 41), dtype=np.uint8)
    assert np.array_equal(crc.remainder_bitwise(m, crc.POLY_B), crc.remainder_table(m, crc.POLY_B))
    word = tx.crc24_attach(m, tx.CRC24B_POLY)
    assert np.array_equal(word[:, m.shape[1]:], crc.crc_bits(m, crc.POLY_B))
    assert np.all(crc.cb_ok(word) == 1)
    word[4, 100] ^= 1
    assert crc.cb_ok(word)[4] == 0


@pytest.fixture(scope="module")
def seg_noiseless():
    return segmented(n_tb=8, noiseless=True)


def test_segmentation_layout(seg_noiseless):
    w = seg_noiseless
    for tb in w.tbs:
        first, n = int(tb["first_cb"]), int(tb["n_cb"])
        assert n >= 2
        Ks = [w.bgs[int(w.cbs[i]["bg"])].kb * int(w.cbs[i]["Z"]) for i in range(first, first + n)]
        assert int(tb["payload_bits"]) == sum(K - 24 for K in Ks) - 24
        assert all(int(w.cbs[i]["flags"]) == 1 for i in range(first, first + n))
    # the transmitted information words: every code block passes its CRC, every TB its own
    d, _, _, _ = goodput.tb_crc_goodput(w, w.info_words)
    assert np.all(d == 1)
    for i in range(w.n_cb):
        assert crc.cb_ok(goodput.cb_bits(w, w.info_words, i))[0] == 1


def test_cb_crc_bits_are_excluded_from_the_tb_check(seg_noiseless):
    w = seg_noiseless
    tb = w.tbs[0]
    i = int(tb["first_cb"])
    K = w.bgs[int(w.cbs[i]["bg"])].kb * int(w.cbs[i]["Z"])
    o = int(w.cbs[i]["bits_word_offset"])

    def flipped(bit):
        words = w.info_words.copy()
        words[o + bit // 32] ^= np.uint32(1 << (bit % 32))
        return words

    # a data bit: both the CB CRC and the TB CRC fail
    words = flipped(7)
    assert crc.cb_ok(goodput.cb_bits(w, words, i))[0] == 0
    assert crc.tb_ok(goodput.tb_bitstream(w, words, 0)[None, :])[0] == 0
    assert goodput.tb_crc_goodput(w, words)[0][0] == 0
    # a CB CRC bit: the TB's own CRC still passes (those bits are not in its stream), yet d_e = 0
    words = flipped(K - 3)
    assert crc.tb_ok(goodput.tb_bitstream(w, words, 0)[None, :])[0] == 1
    assert crc.cb_ok(goodput.cb_bits(w, words, i))[0] == 0
    d = goodput.tb_crc_goodput(w, words)[0]
    assert d[0] == 0 and np.all(d[1:] == 1)


def test_noiseless_segmented_decodes_exactly(seg_noiseless):
    w = seg_noiseless
    llr = demap.demap_workload(w)
    words, status = decoder.decode_workload(w, llr, 10, True)
    assert np.array_equal(words, w.info_words)
    assert np.all((status >> 17) & 1 == 1)
    assert np.all(goodput.tb_crc_goodput(w, words)[0] == 1)


def _flags_off(w):
    cbs = w.cbs.copy()
    cbs["flags"] = 0
    return type(w)(w.name, w.bgs, w.z_set, cbs, w.tbs, w.slot_N, w.sym, w.mask, w.info_words, w.llr_len,
                   w.bits_words, w.snr_db, dict(w.meta))


def test_crc_aided_exit_never_later_and_only_on_a_passing_crc():
    # The decoding trajectory is the same until a block stops; the CRC only adds a reason to stop.
    w = segmented(n_tb=10, spread_db=(-2.0, 0.5))
    llr = demap.demap_workload(w)
    wc, sc = decoder.decode_workload(w, llr, 10, True)
    ws, ss = decoder.decode_workload(_flags_off(w), llr, 10, True)
    it_c, it_s = sc & 0xFFFF, ss & 0xFFFF
    assert np.all(it_c <= it_s)
    assert np.all(((ss >> 17) & 1) == 0)
    earlier = np.flatnonzero(it_c < it_s)
    same = np.flatnonzero(it_c == it_s)
    assert earlier.size > 0  # the CRC exit does fire on these inputs
    for i in earlier:  # stopped by the CRC alone
        assert (sc[i] >> 17) & 1 == 1 and (sc[i] >> 16) & 1 == 0
    for i in range(w.n_cb):
        b = goodput.cb_bits(w, wc, i)
        assert crc.cb_ok(b)[0] == (sc[i] >> 17) & 1
    for i in same:
        o = int(w.cbs[i]["bits_word_offset"])
        K = w.bgs[int(w.cbs[i]["bg"])].kb * int(w.cbs[i]["Z"])
        assert np.array_equal(wc[o:o + K // 32], ws[o:o + K // 32])
    # some blocks fail outright at these SNRs, some decode
    assert 0 < np.count_nonzero((sc >> 17) & 1) < w.n_cb


def test_int8_decoder_honours_the_crc_exit_too():
    w = segmented(n_tb=6, spread_db=(-1.5, 0.5))
    llr = demap.quantise(demap.demap_workload(w), 4.0, 63)
    wc, sc = decoder.decode_workload(w, llr, 10, True, decoder.INT8)
    ws, ss = decoder.decode_workload(_flags_off(w), llr, 10, True, decoder.INT8)
    assert np.all((sc & 0xFFFF) <= (ss & 0xFFFF))
    for i in range(w.n_cb):
        assert crc.cb_ok(goodput.cb_bits(w, wc, i))[0] == (sc[i] >> 17) & 1
