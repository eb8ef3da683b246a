"""Pins for the oracle's CRC-24 check, goodput (eq. 1), reward (eq. 2) and BLER interval."""
import math
import os

import numpy as np
import pytest

from oracle import crc, goodput, stats
from workload import tx
from workload.configs import CB_DTYPE, TB_DTYPE, Workload
from workload.basegraph import make_base_graph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_crc_remainder_of_codeword_is_zero():
    rng = np.random.default_rng(1)
    msg = rng.integers(0, 2, size=(20, 200), dtype=np.uint8)
    word = np.concatenate([msg, crc.crc_bits(msg)], axis=1)
    assert np.all(crc.remainder_bitwise(word) == 0)
    assert np.all(crc.tb_ok(word) == 1)


def test_crc_linear_and_zero():
    rng = np.random.default_rng(2)
    a = rng.integers(0, 2, size=(10, 96), dtype=np.uint8)
    b = rng.integers(0, 2, size=(10, 96), dtype=np.uint8)
    ra, rb, rab = crc.remainder_bitwise(a), crc.remainder_bitwise(b), crc.remainder_bitwise(a ^ b)
    assert np.array_equal(ra ^ rb, rab)
    assert crc.remainder_bitwise(np.zeros((1, 64), np.uint8))[0] == 0


def test_crc_generator_is_a_codeword():
    # g(x) itself, as a 25-bit word (x^24 first), leaves remainder 0.
    g = (1 << 24) | crc.POLY
    bits = np.array([(g >> (24 - i)) & 1 for i in range(25)], dtype=np.uint8)
    assert crc.remainder_bitwise(bits)[0] == 0
    # and a single x^k with k < 24 never does
    for k in range(24):
        e = np.zeros(24, np.uint8)
        e[23 - k] = 1
        assert crc.remainder_bitwise(e)[0] != 0


def test_crc_detects_every_burst_up_to_24():
    rng = np.random.default_rng(3)
    A = 40
    msg = rng.integers(0, 2, size=(1, A), dtype=np.uint8)
    word = np.concatenate([msg, crc.crc_bits(msg)], axis=1)[0]
    n = word.size
    errs = []
    for length in range(1, 25):
        for start in range(0, n - length + 1):
            # bursts: first and last bit of the span set, interior patterns sampled
            for _ in range(2 if length > 2 else 1):
                e = np.zeros(n, np.uint8)
                e[start] = 1
                e[start + length - 1] = 1
                if length > 2:
                    e[start + 1:start + length - 1] = rng.integers(0, 2, size=length - 2)
                errs.append(word ^ e)
    errs = np.array(errs)
    assert np.all(crc.remainder_bitwise(errs) != 0)


def test_crc_bitwise_matches_table():
    rng = np.random.default_rng(4)
    m = rng.integers(0, 2, size=(16, 8 * 37), dtype=np.uint8)
    assert np.array_equal(crc.remainder_bitwise(m), crc.remainder_table(m))


def test_transmitter_crc_agrees_with_oracle_check():
    # two independent CRC implementations: the transmitter's (matrix of x^k mod g)
    # and the oracle's long division.
    rng = np.random.default_rng(5)
    payload = rng.integers(0, 2, size=(8, 104), dtype=np.uint8)
    word = tx.crc24_attach(payload)
    assert np.array_equal(word[:, 104:], crc.crc_bits(payload))
    assert np.all(crc.tb_ok(word) == 1)
    word[3, 17] ^= 1
    assert crc.tb_ok(word)[3] == 0


def _read_golden():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "tti300_goodput_reward.txt"))
            if ln.strip() and not ln.startswith("#")]
    N = int(rows[0][0])
    s = [int(x) for x in rows[1]]
    cases = [(r[0], [int(x) for x in r[1:11]], int(r[11]), int(r[12])) for r in rows[2:]]
    return N, s, cases


def _slot_workload(n_sc, N, d):
    """A one-slot workload whose TB t decodes (CRC ok) iff d[t]: one tiny code block per TB."""
    bg = make_base_graph("tiny")
    Z = 16
    K = bg.kb * Z
    nt = len(n_sc)
    cbs = np.zeros(nt, dtype=CB_DTYPE)
    tbs = np.zeros(nt, dtype=TB_DTYPE)
    words = np.zeros(nt * K // 32, dtype=np.uint32)
    rng = np.random.default_rng(9)
    for t in range(nt):
        cbs[t] = (0, Z, 2, 256, 0, 0, 0, t * K // 32, 1.0, 0)
        tbs[t] = (t, 1, n_sc[t], 0, K - 24)
        payload = rng.integers(0, 2, size=(1, K - 24), dtype=np.uint8)
        bits = np.concatenate([payload, crc.crc_bits(payload)], axis=1)[0]
        if not d[t]:
            bits[5] ^= 1
        words[t * K // 32:(t + 1) * K // 32] = (bits.reshape(-1, 32).astype(np.uint64)
                                                << np.arange(32, dtype=np.uint64)).sum(1).astype(np.uint32)
    return Workload("slot", [bg], [Z], cbs, tbs, np.array([N], np.int32), None, None, None, 0,
                    words.size), words


def test_goodput_reward_tti300_worked_example():
    N, s, cases = _read_golden()
    assert sum(s) == N
    for name, d, g_sc, fail_sc in cases:
        w, words = _slot_workload(s, N, d)
        dd, gb, gs, r = goodput.tb_crc_goodput(w, words)
        assert list(dd) == d, name
        assert gs[0] == g_sc, name
        assert math.isclose(r[0], -fail_sc / N, rel_tol=0, abs_tol=1e-15), name
        assert gb[0] == sum(di * (16 * 8 - 24) for di in d)
        assert -1.0 <= r[0] <= 0.0
    # bounds stated with eq. 2: 0 when all decode, -1 when all fail and sum n_e = N
    assert goodput.reward_closed_form([1] * 10, s, N) == 0.0
    assert goodput.reward_closed_form([0] * 10, s, N) == -1.0


def test_wilson_textbook_values():
    # 0 failures in 10: upper bound z^2 / (n + z^2)
    lo, hi = stats.wilson(0, 10)
    z2 = stats.Z95 ** 2
    assert lo == 0.0 and math.isclose(hi, z2 / (10 + z2), rel_tol=1e-12)
    # symmetric: k and n-k mirror around 1/2
    lo1, hi1 = stats.wilson(3, 20)
    lo2, hi2 = stats.wilson(17, 20)
    assert math.isclose(lo1, 1 - hi2, rel_tol=1e-12) and math.isclose(hi1, 1 - lo2, rel_tol=1e-12)
    # contains the point estimate and shrinks with n
    for k, n in [(5, 50), (50, 500)]:
        lo, hi = stats.wilson(k, n)
        assert lo < k / n < hi
    assert (stats.wilson(50, 500)[1] - stats.wilson(50, 500)[0]) < (stats.wilson(5, 50)[1] - stats.wilson(5, 50)[0])


def test_clopper_pearson_covers_wilson_point():
    pytest.importorskip("scipy")
    lo, hi = stats.clopper_pearson(5, 50)
    assert lo < 0.1 < hi
