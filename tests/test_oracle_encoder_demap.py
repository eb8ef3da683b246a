"""Pins for the base matrices, the oracle encoder and the oracle demapper."""
import numpy as np
import pytest

from oracle import demap, encoder
from workload import tx
from workload.basegraph import make_base_graph, tree_base_graph

# SHA-256 of the seeded base matrices (frozen: any change to the construction or
# the RNG changes them, and every stored expectation with them).
FROZEN_SHA = {
    "bg1": "205c72fcb0589dfb",
    "bg2": "7907f3900d0ca440",
    "tiny": "8d0399c52c209046",
}


@pytest.mark.parametrize("name", ["bg1", "bg2", "tiny"])
def test_base_graph_frozen_and_structured(name):
    bg = make_base_graph(name)
    assert bg.sha256()[:16] == FROZEN_SHA[name]
    assert make_base_graph(name).sha256() == bg.sha256()  # deterministic
    D = bg.dense()
    kb, mc = bg.kb, bg.mc
    # dual diagonal in the core rows (extension rows may also use core parity
    # columns): column kb at rows 0, mc//2, mc-1 with shifts 1, 0, 1
    col = D[:mc, kb]
    assert set(np.flatnonzero(col >= 0)) == {0, mc // 2, mc - 1}
    assert col[0] == 1 and col[mc // 2] == 0 and col[mc - 1] == 1
    for i in range(1, mc):
        assert D[i - 1, kb + i] == 0 and D[i, kb + i] == 0
        assert np.count_nonzero(D[:mc, kb + i] >= 0) == 2
    # extension rows: identity on their own column, nothing else in it
    for r in range(mc, bg.mb):
        assert D[r, kb + r] == 0 and np.count_nonzero(D[:, kb + r] >= 0) == 1
        assert D[r, 0] >= 0 or D[r, 1] >= 0
    # every information column has degree >= 2
    assert np.all((D[:, :kb] >= 0).sum(axis=0) >= 2)
    assert bg.row_degrees().max() <= 27 and bg.row_degrees().min() >= 2


@pytest.mark.parametrize("name,Z", [("tiny", 16), ("tiny", 4), ("bg2", 8), ("bg1", 8), ("bg1", 32)])
def test_encoder_parity_checks_hold(name, Z):
    bg = make_base_graph(name)
    rng = np.random.default_rng(Z)
    for _ in range(3 if Z > 16 else 10):
        u = rng.integers(0, 2, size=bg.kb * Z, dtype=np.uint8)
        c = encoder.encode_one(bg, Z, u)
        assert np.array_equal(c[:bg.kb * Z], u)
        assert not encoder.syndrome(bg, Z, c).any()


def test_encoder_linear_and_matches_transmitter():
    bg = make_base_graph("bg2")
    Z = 16
    rng = np.random.default_rng(7)
    u = rng.integers(0, 2, size=(4, bg.kb * Z), dtype=np.uint8)
    c_or = np.stack([encoder.encode_one(bg, Z, x) for x in u])
    c_tx = tx.encode(bg, Z, u)
    assert np.array_equal(c_or, c_tx)
    assert np.array_equal(encoder.encode_one(bg, Z, u[0] ^ u[1]), c_or[0] ^ c_or[1])
    # a single flipped bit breaks some check
    bad = c_or[0].copy()
    bad[5] ^= 1
    assert encoder.syndrome(bg, Z, bad).any()


def test_qpsk_closed_form():
    rng = np.random.default_rng(0)
    y = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    s2 = 0.37
    lam = demap.maxlog_llr(y, 2, 1.0 / s2)
    assert np.allclose(lam[:, 0], 2 * np.sqrt(2) * y.real / s2, rtol=1e-12, atol=1e-12)
    assert np.allclose(lam[:, 1], 2 * np.sqrt(2) * y.imag / s2, rtol=1e-12, atol=1e-12)


def test_16qam_amplitude_bit_closed_form():
    # I-axis amplitude bit b2 of 16-QAM: levels |1| (b2=0) and |3| (b2=1), /sqrt(10).
    # For y_I = u / sqrt(10) with 1 <= u <= 3: lambda = ((u-3)^2 - (u-1)^2) / (10 s2) = (8 - 4u) / (10 s2)
    s2 = 0.5
    u = np.linspace(1.0, 3.0, 9)
    y = u / np.sqrt(10) + 0.2j / np.sqrt(10)
    lam = demap.maxlog_llr(y, 4, 1.0 / s2)
    assert np.allclose(lam[:, 2], (8 - 4 * u) / (10 * s2), atol=1e-12)
    # sign bit b0 there: nearest b0=1 level is -1; nearest b0=0 level is 1 for
    # u <= 2 and 3 beyond, so lambda = 4u/(10 s2) for u <= 2, (8u - 8)/(10 s2) above
    want = np.where(u <= 2, 4 * u, 8 * u - 8) / (10 * s2)
    assert np.allclose(lam[:, 0], want, atol=1e-12)


@pytest.mark.parametrize("Qm", [2, 4, 6, 8])
def test_demap_symmetry_and_noiseless_signs(Qm):
    rng = np.random.default_rng(Qm)
    pts, labels = demap.constellation(Qm)
    assert np.isclose(np.mean(np.abs(pts) ** 2), 1.0)
    # transmitter mapping agrees with the oracle constellation
    assert np.allclose(tx.qam_map(labels), pts)
    lam = demap.maxlog_llr(pts, Qm, 1.0)
    assert np.array_equal(lam < 0, labels.astype(bool))
    y = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    a, b = demap.maxlog_llr(y, Qm, 1.0), demap.maxlog_llr(-y, Qm, 1.0)
    assert np.allclose(a[:, :2], -b[:, :2])      # sign-carrying bits: odd
    assert np.allclose(a[:, 2:], b[:, 2:])       # amplitude bits: even


@pytest.mark.parametrize("Qm", [4, 6, 8])
def test_demap_separable_equals_two_dimensional(Qm):
    # per-axis minimum over the PAM levels, written from the definition, equals
    # the 2-D brute force the oracle runs.
    rng = np.random.default_rng(10 + Qm)
    y = 1.3 * (rng.standard_normal(64) + 1j * rng.standard_normal(64))
    full = demap.maxlog_llr(y, Qm, 2.0)
    pts, labels = demap.constellation(Qm)
    sep = np.zeros_like(full)
    for i in range(Qm):
        comp = y.real if i % 2 == 0 else y.imag
        lv = (pts.real if i % 2 == 0 else pts.imag)
        d = (comp[:, None] - lv[None, :]) ** 2
        one = labels[:, i] == 1
        sep[:, i] = 2.0 * (d[:, one].min(1) - d[:, ~one].min(1))
    assert np.allclose(full, sep, atol=1e-12)


def test_demap_flush_and_positions():
    bg = make_base_graph("bg2")
    Z, Qm, E = 32, 4, 4 * 100
    rng = np.random.default_rng(3)
    y = rng.standard_normal(E // Qm) + 1j * rng.standard_normal(E // Qm)
    mask = np.zeros(E // Qm, bool)
    mask[[0, 7, 99]] = True
    out = demap.demap_cb(y, mask, bg, Z, Qm, E, 1.0)
    t0, m_eff, n_eff = demap.bg_geometry(bg, Z, E)
    assert t0 == 64 and out.size == n_eff * Z
    assert np.all(out[:t0] == 0) and np.all(out[t0 + E:] == 0)
    lam = demap.maxlog_llr(y, Qm, 1.0)
    n_re = E // Qm
    for r in [1, 50]:
        for i in range(Qm):
            assert out[t0 + i * n_re + r] == lam[r, i]
    for r in [0, 7, 99]:
        assert all(out[t0 + i * n_re + r] == 0 for i in range(Qm))


def test_quantiser_rounds_half_away_and_saturates():
    x = np.array([0.124, 0.125, -0.125, 0.375, -0.376, 100.0, -100.0, 0.0])
    q = demap.quantise(x, 4.0, 63)
    assert list(q) == [0, 1, -1, 2, -2, 63, -63, 0]


def test_geometry_large_code():
    bg = make_base_graph("bg1")
    assert demap.bg_geometry(bg, 384, 16896) == (768, 24, 46)
    tiny = make_base_graph("tiny")
    assert demap.bg_geometry(tiny, 16, 256) == (0, 8, 16)
    # same geometry from the workload's helpers (two independent formulas)
    assert (bg.t0(384), bg.m_eff(384, 16896), bg.n_eff(384, 16896)) == (768, 24, 46)
    assert tree_base_graph().n_edges == 9


def test_rate_matching_wraps_the_circular_buffer():
    from workload import tx as TX
    from workload import default_bgs
    bgs = default_bgs()
    bg, Z = bgs[0], 64
    rng = np.random.default_rng(3)
    info = rng.integers(0, 2, size=(2, bg.kb * Z), dtype=np.uint8)
    cw = TX.encode(bg, Z, info, n_cols=bg.nb)
    ncb = bg.nb * Z - bg.t0(Z)
    E = ncb + 500
    e = TX.rate_match(bg, Z, cw, E)
    assert np.array_equal(e[:, :ncb], cw[:, bg.t0(Z):]) and np.array_equal(e[:, ncb:], e[:, :500])


def test_repeated_positions_add_their_llrs():
    # noiseless QPSK at unit 1/sigma^2: every bit's max-log LLR is +-2 (2 sqrt2 * 1/sqrt2); a position sent
    # twice carries the sum, +-4, with the sign of its bit
    from workload import tx as TX
    from workload import default_bgs
    bgs = default_bgs()
    bg, Z, Qm = bgs[1], 32, 2
    ncb = bg.nb * Z - bg.t0(Z)
    E = ncb + 2 * 150
    rng = np.random.default_rng(4)
    info = rng.integers(0, 2, size=(1, bg.kb * Z), dtype=np.uint8)
    cw = TX.encode(bg, Z, info, n_cols=bg.nb)
    y = TX.qam_map(TX.interleave(TX.rate_match(bg, Z, cw, E), Qm, True))[0]
    llr = demap.demap_cb(y, np.zeros(E // Qm, dtype=bool), bg, Z, Qm, E, 1.0, True)
    t0 = bg.t0(Z)
    sign = 1.0 - 2.0 * cw[0, t0:].astype(np.float64)
    assert np.allclose(llr[t0:t0 + 300], 4.0 * sign[:300], atol=1e-9)
    assert np.allclose(llr[t0 + 300:t0 + ncb], 2.0 * sign[300:ncb], atol=1e-9)
    assert np.all(llr[:t0] == 0)


def test_noiseless_repetition_decodes_exactly():
    from oracle import path as opath
    from workload.configs import repetition
    w = repetition(3, noiseless=True)
    assert np.all(w.cbs["E"] > np.array([w.bgs[int(c["bg"])].nb * int(c["Z"]) - w.bgs[int(c["bg"])].t0(int(c["Z"]))
                                         for c in w.cbs]))
    r = opath.run(w, "f64", 10, True)
    assert opath.block_errors(w, r["words"]).sum() == 0 and np.all(r["d"] == 1)
