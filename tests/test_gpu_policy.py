"""Puncturing allocations on the GPU (RP, SeF, feasibility enforcer, SC masks) against the oracle, bit for bit."""
import numpy as np
import pytest
import torch

from oracle import policy as P
from paper_2506_00167_gb300 import policy as G

pytestmark = pytest.mark.gpu


def _cuda_i32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _oracle_alloc(alloc, demand, policy):
    T, E = alloc.shape
    out = np.zeros((T, 7, E), dtype=np.int64)
    st = np.zeros((T, 7), dtype=np.int64)
    fn = {"rp": P.rp, "sef": P.sef}[policy]
    for t in range(T):
        for ms in range(7):
            d = int(demand[t, ms])
            if d > alloc[t].sum():
                st[t, ms] = 1
            elif d:
                out[t, ms] = fn(alloc[t], d)
    return out, st


def test_table6_tti():
    s = np.array([[60, 108, 72, 72, 72, 48, 72, 48, 96, 132]])
    demand = np.array([[0, 300, 0, 0, 300, 0, 600]])
    for policy in ["rp", "sef"]:
        m, st = G.puncture_alloc(_cuda_i32(s), _cuda_i32(demand), policy)
        want, wst = _oracle_alloc(s, demand, policy)
        assert np.array_equal(m.cpu().numpy(), want) and np.array_equal(st.cpu().numpy(), wst)
    m, _ = G.puncture_alloc(_cuda_i32(s), _cuda_i32(demand), "rp")
    assert m[0, 1].tolist() == [23, 41, 28, 28, 28, 18, 28, 18, 37, 51]   # Table VI, RP, 300 SCs


@pytest.mark.parametrize("E", [1, 10, 32])
@pytest.mark.parametrize("policy", ["rp", "sef"])
def test_alloc_matches_oracle(E, policy):
    rng = np.random.default_rng(100 + E)
    T = 600
    alloc = rng.integers(12, 200, size=(T, E))
    alloc[::7] = 48                                   # ties everywhere
    tot = alloc.sum(axis=1, keepdims=True)
    demand = (rng.random((T, 7)) * 1.1 * tot).astype(np.int64)
    demand[rng.random((T, 7)) < 0.3] = 0
    demand[::11, 3] = tot[::11, 0]                    # whole slot punctured
    m, st = G.puncture_alloc(_cuda_i32(alloc), _cuda_i32(demand), policy)
    want, wst = _oracle_alloc(alloc, demand, policy)
    assert np.array_equal(st.cpu().numpy(), wst) and wst.any()
    assert np.array_equal(m.cpu().numpy(), want)


def _oracle_enforce(mr, n, total):
    out = np.zeros(n.shape, dtype=np.int64)
    st = np.zeros(len(total), dtype=np.int64)
    for p in range(len(total)):
        try:
            x = P.kl_project(mr[p], n[p], int(total[p]))
        except ValueError:
            st[p] = 1
            continue
        try:
            out[p] = P.hh_round(x, int(total[p]), n[p])
        except ValueError:
            st[p] = 2
    return out, st


@pytest.mark.parametrize("E", [1, 10, 32])
def test_enforcer_matches_oracle(E):
    rng = np.random.default_rng(200 + E)
    Pn = 3000
    n = rng.integers(12, 150, size=(Pn, E))
    mr = (rng.uniform(0, 1.6, size=(Pn, E)) * n).astype(np.float32)
    mr[rng.random((Pn, E)) < 0.2] = 0.0              # users the policy leaves alone
    mr[::5] = np.round(mr[::5])                       # integer-valued inputs, ties among breakpoints
    mr[::13, : max(1, E // 2)] = -1.0                 # negative entries count as zero
    L = rng.integers(20, 300, size=Pn)
    j = np.maximum(1, (rng.random(Pn) * (n.sum(axis=1) // L + 1)).astype(np.int64))
    total = j * L
    total[::17] = n.sum(axis=1)[::17] + 1             # infeasible on purpose
    out, st = G.enforce(torch.from_numpy(mr).cuda(), _cuda_i32(n), _cuda_i32(total))
    want, wst = _oracle_enforce(mr, n, total)
    got_st = st.cpu().numpy()
    assert np.array_equal(got_st, wst) and (wst == 1).any()
    assert np.array_equal(out.cpu().numpy(), want)
    ok = got_st == 0
    o = out.cpu().numpy()
    assert np.array_equal(o[ok].sum(axis=1), total[ok]) and np.all(o[ok] <= n[ok]) and np.all(o >= 0)


def test_sc_mask_matches_oracle():
    rng = np.random.default_rng(300)
    T, E = 400, 10
    alloc = rng.integers(12, 132, size=(T, E))
    demand = (rng.random((T, 7)) * alloc.sum(axis=1, keepdims=True)).astype(np.int64)
    demand[rng.random((T, 7)) < 0.4] = 0
    m, _ = G.puncture_alloc(_cuda_i32(alloc), _cuda_i32(demand), "rp")
    words = (int(alloc.sum(axis=1).max()) + 31) // 32
    mask = G.sc_mask(_cuda_i32(alloc), m, words).cpu().numpy().view(np.uint32)
    mnp = m.cpu().numpy()
    for t in range(0, T, 7):
        want = P.sc_mask(alloc[t], mnp[t])                        # (14, sum(n)) bool
        bits = np.unpackbits(mask[t].astype("<u4").view(np.uint8), bitorder="little").reshape(14, words * 32)
        assert np.array_equal(bits[:, : want.shape[1]].astype(bool), want)
        assert not bits[:, want.shape[1]:].any()


def test_rt_odu_codebook_matches_oracle():
    from workload.policy import actor_noise, actor_weights, schedules
    T = 300
    alloc, _ = schedules(T, seed=41)
    w1, b1, w2, b2 = actor_weights(seed=42)
    noise = actor_noise(T, seed=43)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    book, act, st = G.rt_odu_codebook(_cuda_i32(alloc), cu(w1), cu(b1), cu(w2), cu(b2), cu(noise), 300)
    book, act, st = book.cpu().numpy(), act.cpu().numpy(), st.cpu().numpy()
    assert not st.any()
    same = 0
    for t in range(T):
        wb, wa = P.rt_odu_codebook(alloc[t], w1, b1, w2, b2, noise[t], 300)
        # tanh/exp/log1p of the GPU and of NumPy may differ in the last bit: actions agree to float32
        # rounding, codebooks exactly unless a Huntington-Hill priority falls on such a difference
        assert np.allclose(act[t], wa, rtol=2e-6, atol=1e-7)
        same += int(np.array_equal(book[t], wb))
        for j in range(book.shape[1]):
            assert book[t, j].sum() == 300 * (j + 1) and np.all(book[t, j] <= alloc[t]) and np.all(book[t, j] >= 0)
    assert same >= 0.99 * T


def test_rt_odu_uniform_policy_is_rp_bit_exact():
    s = np.array([[60, 108, 72, 72, 72, 48, 72, 48, 96, 132]])
    E, H = 10, 128
    z = lambda *sh: torch.zeros(sh, dtype=torch.float32, device="cuda")
    b2 = z(2 * E)
    b2[:E] = 0.3
    book, _, st = G.rt_odu_codebook(_cuda_i32(s), z(H, E + 1), z(H), z(2 * E, H), b2, z(1, 2, E), 300)
    assert not st.any()
    assert book[0, 0].tolist() == P.rp(s[0], 300).tolist() and book[0, 1].tolist() == P.rp(s[0], 600).tolist()
