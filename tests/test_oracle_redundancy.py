"""Pins for redundancy versions 1-3: where each version starts in the circular buffer, how the versions
tile it, the oracle's dematching against the transmitter's rate matching, and noiseless decoding of the
self-decodable versions."""
import numpy as np
import pytest

from oracle import decoder, demap
from workload import default_bgs
from workload import tx as TX
from workload.configs import cb_rv, redundancy_versions


@pytest.mark.parametrize("b", [0, 1])
def test_version_two_starts_mid_buffer_and_starts_increase(b):
    bg = default_bgs()[b]
    for Z in (32, 64, 384):
        ncb = bg.ncb(Z)
        k = [bg.k0(Z, rv) for rv in range(4)]
        assert k[0] == 0 and k[2] == ncb // 2          # the middle of the buffer, both graph sizes
        assert k == sorted(k) and k[3] < ncb and all(x % Z == 0 for x in k)
        assert k == [demap.start_k0(bg.nb, bg.n_punct_cols, Z, rv) for rv in range(4)]


def test_other_graphs_accept_version_zero_only():
    tiny = default_bgs()[2]
    assert tiny.k0(16, 0) == 0
    with pytest.raises(ValueError):
        tiny.k0(16, 1)
    with pytest.raises(ValueError):
        demap.start_k0(tiny.nb, tiny.n_punct_cols, 16, 2)


@pytest.mark.parametrize("b", [0, 1])
def test_versions_read_one_circular_buffer(b):
    # version rv sends the buffer from k0(rv) on: its first k0(rv+1) - k0(rv) bits are the bits of
    # version 0 at those offsets, and E = Ncb from any start visits every position exactly once
    bg, Z = default_bgs()[b], 32
    rng = np.random.default_rng(30 + b)
    info = rng.integers(0, 2, size=(2, bg.kb * Z), dtype=np.uint8)
    cw = TX.encode(bg, Z, info, n_cols=bg.nb)
    ncb = bg.ncb(Z)
    whole = TX.rate_match(bg, Z, cw, ncb, 0)
    assert np.array_equal(whole, cw[:, bg.t0(Z):])
    for rv in range(1, 4):
        k0 = bg.k0(Z, rv)
        e = TX.rate_match(bg, Z, cw, ncb, rv)
        assert np.array_equal(e, np.roll(whole, -k0, axis=1))
        n = (bg.k0(Z, rv + 1) if rv < 3 else ncb) - k0
        assert np.array_equal(e[:, :n], whole[:, k0:k0 + n])


@pytest.mark.parametrize("rv", [0, 1, 2, 3])
def test_dematching_puts_each_bit_where_the_transmitter_sent_it(rv):
    # noiseless QPSK, 1/sigma^2 = 1: every sent bit's LLR is +-2 with its codeword bit's sign, a position
    # sent twice +-4, a position never sent 0 -- the oracle's dematching against the transmitter's
    bg, Z, Qm = default_bgs()[0], 32, 2
    ncb = bg.ncb(Z)
    rng = np.random.default_rng(40 + rv)
    info = rng.integers(0, 2, size=(1, bg.kb * Z), dtype=np.uint8)
    cw = TX.encode(bg, Z, info, n_cols=bg.nb)
    for E in (ncb // 2, ncb - 2 * Z, ncb + 6 * Z):
        y = TX.qam_map(TX.interleave(TX.rate_match(bg, Z, cw, E, rv), Qm, True))[0]
        llr = demap.demap_cb(y, np.zeros(E // Qm, dtype=bool), bg, Z, Qm, E, 1.0, True, rv)
        t0 = bg.t0(Z)
        hits = np.zeros(bg.nb * Z, dtype=np.int64)
        np.add.at(hits, t0 + (bg.k0(Z, rv) + np.arange(E)) % ncb, 1)
        sign = 1.0 - 2.0 * cw[0].astype(np.float64)
        n = llr.size
        assert np.allclose(llr, 2.0 * hits[:n] * sign[:n], atol=1e-9)
        assert hits[n:].sum() == 0  # nothing is sent beyond the decoded columns


def test_geometry_follows_the_last_position_sent():
    bg = default_bgs()[0]
    Z, E = 64, 44 * 64                      # rate 1/2: 44 Z bits
    assert demap.bg_geometry(bg, Z, E, 0) == (128, 24, 46)
    assert demap.bg_geometry(bg, Z, E, 1) == (128, 41, 63)   # 17 Z + 44 Z = 61 Z: columns up to 62
    assert demap.bg_geometry(bg, Z, E, 2)[1:] == (46, 68)    # 33 Z + 44 Z wraps the 66 Z buffer
    for rv in range(4):
        assert demap.bg_geometry(bg, Z, E, rv)[1] == bg.m_eff(Z, E, rv)


def test_self_decodable_versions_decode_noiseless():
    # versions 0 and 3 carry enough systematic bits to decode alone at these rates
    w = redundancy_versions(n_per=1, noiseless=True)
    llr = demap.demap_workload(w)
    words, status = decoder.decode_workload(w, llr, 10, True)
    seen = set()
    for i in range(w.n_cb):
        c = w.cbs[i]
        rv = cb_rv(c)
        seen.add(rv)
        if rv in (0, 3):
            K = w.bgs[int(c["bg"])].kb * int(c["Z"])
            o = int(c["bits_word_offset"])
            assert np.array_equal(words[o:o + K // 32], w.info_words[o:o + K // 32]), i
            assert (status[i] >> 16) & 1 == 1
    assert seen == {0, 1, 2, 3}
