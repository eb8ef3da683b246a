"""GPU parity: every step of the CUDA path against the CPU oracle on the same seeded inputs.

Bars: integer decode bit-exact (bits, iteration counts, syndrome flags);
float32 decode bit-exact against the oracle's float32 run and >= 99.9 % of
code blocks identical to its float64 run; demapped LLRs within
1e-4 * max(|lambda|, 1) of the float64 oracle, punctured LLRs exactly 0;
quantised LLRs within 1 LSB everywhere; CRC flags and goodput exact, reward
within one float32 ulp.
"""
import numpy as np
import pytest
import torch

from oracle import decoder as odec
from oracle import demap as odemap
from oracle import goodput as ogood
from oracle import path as opath
from workload import large_fp32, mixed, tiny_fp32
from workload.configs import redundancy_versions, repetition, segmented
from workload.basegraph import tree_base_graph

from gpu_helpers import LLR_NP, batch_for, device_inputs, session_for, to_np_u32

pytestmark = pytest.mark.gpu

ARITH = {"f32": odec.F32, "i8": odec.INT8, "i16": odec.INT16}
QUANT = {"i8": (4.0, 63), "i16": (4.0, 1023)}


def _workloads():
    return {
        "tiny": tiny_fp32(n_per_point=24, ebn0_points=(1, 3)),
        "large": large_fp32(n_cw=10, snr_points=(6, 8, 10, 12)),
        "mixed": mixed(n_slots=3, ues_per_slot=4, max_cb=3),
        "repetition": repetition(n_per_shape=8),   # rate matching wraps the circular buffer
        # segmented TBs with a CRC per code block: CRC-aided exit and the segmented TB check
        "segmented": segmented(n_tb=12, spread_db=(-2.0, 1.0)),
        "mixed_seg": mixed(n_slots=3, ues_per_slot=4, max_cb=3, cb_crc=True, spread_db=2.0),
        # redundancy versions 0-3: buffer starts inside the buffer, wraps, repetition
        "redundancy": redundancy_versions(n_per=2, rates=(0.5, 0.3, 0.2)),
    }


@pytest.fixture(scope="module")
def wls():
    return _workloads()


def _oracle_llr_for_mode(w, mode):
    llr = odemap.demap_workload(w)
    if mode == "f32":
        return llr.astype(np.float32)
    sc, sat = QUANT[mode]
    return odemap.quantise(llr, sc, sat)


def _params(w):
    return w.meta["max_iter"], bool(w.meta["early_term"])


# ------------------------------------------------------------------ demap
@pytest.mark.parametrize("name", ["tiny", "large", "mixed", "repetition", "redundancy"])
def test_demap_f32_matches_oracle(wls, name):
    w = wls[name]
    s = session_for(w, "f32")
    b = batch_for(s, w, with_tbs=False)
    sym, mask = device_inputs(w)
    llr = torch.full((b.info.llr_elems,), 7.0, dtype=torch.float32, device="cuda")  # poison
    s.puncture_demap(b, sym, mask, llr)
    torch.cuda.synchronize()
    got = llr.cpu().numpy().astype(np.float64)
    want = odemap.demap_workload(w)
    tol = 1e-4 * np.maximum(np.abs(want), 1.0)
    assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want) / tol)
    assert np.array_equal(got == 0.0, want == 0.0) or np.all(got[want == 0.0] == 0.0)
    assert s.device_errors() == 0


@pytest.mark.parametrize("mode", ["i8", "i16"])
@pytest.mark.parametrize("name", ["large", "mixed", "repetition", "redundancy"])
def test_demap_quantised_within_one_lsb(wls, name, mode):
    w = wls[name]
    s = session_for(w, mode)
    b = batch_for(s, w, with_tbs=False)
    sym, mask = device_inputs(w)
    llr = torch.full((b.info.llr_elems,), 5, dtype=getattr(torch, {"i8": "int8", "i16": "int16"}[mode]),
                     device="cuda")
    s.puncture_demap(b, sym, mask, llr)
    got = llr.cpu().numpy().astype(np.int64)
    want = _oracle_llr_for_mode(w, mode)
    diff = np.abs(got - want)
    assert diff.max() <= 1
    assert np.mean(diff == 0) >= 0.999
    # punctured / never-sent positions are exactly 0 on both sides
    zero = odemap.demap_workload(w) == 0.0
    assert np.all(got[zero] == 0)


# ------------------------------------------------------------------ decode
@pytest.mark.parametrize("mode", ["i8", "i16"])
@pytest.mark.parametrize("name", ["tiny", "large", "mixed", "repetition", "segmented", "mixed_seg", "redundancy"])
def test_decode_integer_bit_exact(wls, name, mode):
    w = wls[name]
    mi, et = _params(w)
    llr_np = _oracle_llr_for_mode(w, mode)
    want_bits, want_status = odec.decode_workload(w, llr_np, mi, et, ARITH[mode])
    s = session_for(w, mode, max_iter=mi, early_term=et)
    b = batch_for(s, w, with_tbs=False)
    llr = torch.from_numpy(llr_np.astype(LLR_NP[mode])).cuda()
    bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
    status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
    s.decode_batch(b, llr, bits, status)
    assert np.array_equal(to_np_u32(bits), want_bits)
    assert np.array_equal(status.cpu().numpy(), want_status)
    assert s.device_errors() == 0


@pytest.mark.parametrize("name", ["tiny", "large", "mixed", "repetition", "segmented", "mixed_seg", "redundancy"])
def test_decode_f32_bit_exact_vs_oracle_float32(wls, name):
    w = wls[name]
    mi, et = _params(w)
    llr_np = _oracle_llr_for_mode(w, "f32")
    want_bits, want_status = odec.decode_workload(w, llr_np, mi, et, odec.F32)
    s = session_for(w, "f32", max_iter=mi, early_term=et)
    b = batch_for(s, w, with_tbs=False)
    bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
    status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
    s.decode_batch(b, torch.from_numpy(llr_np).cuda(), bits, status)
    assert np.array_equal(to_np_u32(bits), want_bits)
    assert np.array_equal(status.cpu().numpy(), want_status)


@pytest.mark.parametrize("name", ["large", "mixed"])
def test_decode_f32_against_float64_oracle(wls, name):
    w = wls[name]
    mi, et = _params(w)
    llr64 = odemap.demap_workload(w)
    want_bits, _ = odec.decode_workload(w, llr64, mi, et, odec.F64)
    s = session_for(w, "f32", max_iter=mi, early_term=et)
    b = batch_for(s, w, with_tbs=False)
    bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
    status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
    s.decode_batch(b, torch.from_numpy(llr64.astype(np.float32)).cuda(), bits, status)
    got = to_np_u32(bits)
    same = []
    for c in w.cbs:
        K = w.bgs[int(c["bg"])].kb * int(c["Z"])
        o = int(c["bits_word_offset"])
        same.append(np.array_equal(got[o:o + K // 32], want_bits[o:o + K // 32]))
    assert np.mean(same) >= 0.999 or sum(not x for x in same) <= 0


# ------------------------------------------------------------------ CRC, goodput, reward
@pytest.mark.parametrize("name", ["tiny", "large", "mixed", "segmented", "mixed_seg"])
def test_crc_goodput_reward_exact(wls, name):
    w = wls[name]
    mi, et = _params(w)
    ref = opath.run(w, "f64", mi, et)
    words = ref["words"].copy()
    # also flip one bit of a few TBs so both outcomes occur
    for t in range(0, w.n_tb, 3):
        o = int(w.cbs[int(w.tbs[t]["first_cb"])]["bits_word_offset"])
        words[o] ^= np.uint32(1 << 7)
    # and, in TBs with code-block CRCs, one CRC bit of their last block (outside the TB's own stream)
    for t in range(1, w.n_tb, 3):
        c = w.cbs[int(w.tbs[t]["first_cb"]) + int(w.tbs[t]["n_cb"]) - 1]
        if int(c["flags"]) & 1:
            K = w.bgs[int(c["bg"])].kb * int(c["Z"])
            words[int(c["bits_word_offset"]) + (K - 5) // 32] ^= np.uint32(1 << ((K - 5) % 32))
    d, gb, gs, r = ogood.tb_crc_goodput(w, words)
    s = session_for(w, "f32")
    b = batch_for(s, w)
    out = b.alloc_outputs()
    bits = torch.from_numpy(words.view(np.int32)).cuda()
    s.tb_crc_goodput(b, bits, out["d"], out["goodput_bits"], out["goodput_sc"], out["reward"])
    assert np.array_equal(out["d"].cpu().numpy()[:w.n_tb], d)
    assert np.array_equal(out["goodput_bits"].cpu().numpy()[:w.n_slots], gb)
    assert np.array_equal(out["goodput_sc"].cpu().numpy()[:w.n_slots], gs)
    rg = out["reward"].cpu().numpy()[:w.n_slots].astype(np.float64)
    assert np.all(np.abs(rg - r) <= np.abs(r) * 2.0 ** -23 + 1e-30)
    assert np.all((rg >= -1.0) & (rg <= 0.0))


# ------------------------------------------------------------------ whole path
@pytest.mark.parametrize("mode", ["f32", "i8"])
@pytest.mark.parametrize("name", ["tiny", "large", "mixed", "mixed_seg", "redundancy"])
def test_full_path_matches_oracle(wls, name, mode):
    # both sides run the whole path from the same symbols and masks; each
    # demaps on its own (float32 here, float64 in the oracle), so a marginal
    # block may decode differently -- TB outcomes must agree on >= 99 %, and
    # the GPU's goodput and reward must follow from its own d_e by eq. 1 / 2.
    w = wls[name]
    mi, et = _params(w)
    s = session_for(w, mode, max_iter=mi, early_term=et)
    b = batch_for(s, w)
    sym, mask = device_inputs(w)
    out = s.run(b, sym, mask, b.alloc_outputs())
    torch.cuda.synchronize()
    ref = opath.run(w, "f32" if mode == "f32" else mode, mi, et)
    d = out["d"].cpu().numpy()[:w.n_tb]
    assert np.mean(d == ref["d"]) >= 0.99
    st = out["status"].cpu().numpy()
    assert np.mean(st == ref["status"]) >= 0.99
    gs = np.zeros(w.n_slots, np.int64)
    fail = np.zeros(w.n_slots, np.int64)
    for t, tb in enumerate(w.tbs):
        gs[tb["slot"]] += int(d[t]) * int(tb["n_sc"])
        fail[tb["slot"]] += (1 - int(d[t])) * int(tb["n_sc"])
    assert np.array_equal(out["goodput_sc"].cpu().numpy()[:w.n_slots], gs)
    r = out["reward"].cpu().numpy()[:w.n_slots]
    assert np.allclose(r, -fail / w.slot_N, rtol=2.0 ** -22, atol=0)
    assert s.device_errors() == 0


# ------------------------------------------------------------------ edge cases
def test_empty_batch_is_a_no_op():
    w = tiny_fp32(n_per_point=2, ebn0_points=(3,))
    s = session_for(w, "f32")
    b = s.batch(w.cbs[:0])
    assert b.info.n_cb == 0
    z = torch.zeros(16, dtype=torch.float32, device="cuda")
    zi = torch.zeros(16, dtype=torch.int32, device="cuda")
    s.decode_batch(b, z, zi, zi)
    s.puncture_demap(b, torch.zeros(4, dtype=torch.complex64, device="cuda"), zi, z)
    assert s.device_errors() == 0


def test_low_rate_z384_uses_global_messages_and_matches():
    # BG1 at the lowest rate: 46 decoded rows at Z=384 -- the float32 state no
    # longer fits shared memory and the check messages live in global scratch.
    from workload.configs import TBSpec, build, default_bgs, es_n0_sigma2
    bgs = default_bgs()
    Z, Qm = 384, 2
    E = (bgs[0].nb - 2) * Z  # every column after the first two is transmitted
    specs = [TBSpec(i, 0, Z, Qm, E, 1, float(es_n0_sigma2(snr)), 0, (E // Qm) // 14 + 1)
             for i, snr in enumerate([-1.0, 0.0, 1.0])]
    punct = [np.zeros((14, sp.width), bool) for sp in specs]
    w = build("lowrate", bgs, specs, [sp.width for sp in specs], punct, seed=77)
    assert w.cb_geometry(0)[3] == 46
    for mode in ["f32", "i16"]:
        llr_np = _oracle_llr_for_mode(w, mode)
        want_bits, want_status = odec.decode_workload(w, llr_np, 10, True, ARITH[mode])
        s = session_for(w, mode, max_iter=10, early_term=True)
        b = s.batch(w.cbs)
        bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
        status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
        s.decode_batch(b, torch.from_numpy(llr_np.astype(LLR_NP[mode])).cuda(), bits, status)
        assert np.array_equal(to_np_u32(bits), want_bits), mode
        assert np.array_equal(status.cpu().numpy(), want_status), mode


def test_tree_code_on_gpu_matches_oracle():
    from workload.configs import TBSpec, build
    bg = tree_base_graph()
    Z = 16
    E = bg.nb * Z
    specs = [TBSpec(i, 0, Z, 2, E, 1, 0.8, 0, 10) for i in range(5)]
    punct = [np.zeros((14, 10), bool) for _ in specs]
    w = build("tree", [bg], specs, [10] * 5, punct, seed=3, z_set=[16])
    llr_np = odemap.demap_workload(w).astype(np.float32)
    want_bits, want_status = odec.decode_workload(w, llr_np, 6, False, odec.F32)
    s = session_for(w, "f32", max_iter=6, early_term=False)
    b = s.batch(w.cbs)
    bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
    status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
    s.decode_batch(b, torch.from_numpy(llr_np).cuda(), bits, status)
    assert np.array_equal(to_np_u32(bits), want_bits)
    assert np.array_equal(status.cpu().numpy(), want_status)


def test_all_zero_llrs_give_zero_word_in_one_iteration():
    w = large_fp32(n_cw=4)
    for mode in ["f32", "i8"]:
        s = session_for(w, mode)
        b = s.batch(w.cbs)
        llr = torch.zeros(b.info.llr_elems, dtype=getattr(torch, {"f32": "float32", "i8": "int8"}[mode]),
                          device="cuda")
        bits = torch.ones(b.info.bits_words, dtype=torch.int32, device="cuda")
        status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
        s.decode_batch(b, llr, bits, status)
        assert int(bits.abs().sum()) == 0
        assert np.all(status.cpu().numpy() == (1 | (1 << 16)))


def test_deterministic_reruns(wls):
    w = wls["mixed"]
    s = session_for(w, "i8")
    b = batch_for(s, w)
    sym, mask = device_inputs(w)
    a = s.run(b, sym, mask, b.alloc_outputs())
    c = s.run(b, sym, mask, b.alloc_outputs())
    for k in ["llr", "bits", "status", "d", "goodput_bits", "reward"]:
        assert torch.equal(a[k], c[k]), k


def test_invalid_descriptors_rejected_on_host():
    from paper_2506_00167_gb300 import LdpcError
    w = large_fp32(n_cw=2)
    s = session_for(w, "f32")
    bad = w.cbs.copy()
    bad["Z"][0] = 48
    with pytest.raises(LdpcError, match="EINVAL"):
        s.batch(bad)
    bad = w.cbs.copy()
    bad["E"][0] = 10 ** 6
    with pytest.raises(LdpcError, match="EINVAL"):
        s.batch(bad)
    bad = w.cbs.copy()
    bad["llr_offset"][1] += 1
    with pytest.raises(LdpcError, match="aligned"):
        s.batch(bad)
    tbs = w.tbs.copy()
    tbs["payload_bits"][0] += 1
    with pytest.raises(LdpcError, match="payload"):
        s.batch(w.cbs, tbs, w.slot_N)


def test_invalid_block_flags_rejected_on_host(wls):
    from paper_2506_00167_gb300 import LdpcError
    w = wls["segmented"]
    s = session_for(w, "f32")
    bad = w.cbs.copy()
    bad["flags"][0] |= 8                                    # no such flag
    with pytest.raises(LdpcError, match="flag"):
        s.batch(bad)
    # a TB whose blocks disagree on carrying a CRC
    bad = w.cbs.copy()
    bad["flags"][int(w.tbs["first_cb"][0])] = 0
    with pytest.raises(LdpcError, match="all or none"):
        s.batch(bad, w.tbs, w.slot_N)
    # payload_bits must account for the block CRCs
    tbs = w.tbs.copy()
    tbs["payload_bits"][0] += 24
    with pytest.raises(LdpcError, match="payload"):
        s.batch(w.cbs, tbs, w.slot_N)
    # redundancy versions 1-3 need a 66 Z or 50 Z buffer: not the tiny graph's
    t = wls["tiny"]
    st = session_for(t, "f32")
    bad = t.cbs.copy()
    bad["flags"][0] = 1 << 1
    with pytest.raises(LdpcError, match="redundancy"):
        st.batch(bad)


def _extreme_degree_graph():
    """4 x 30 base matrix with rows of the largest (27) and smallest (2) degree the decoders accept, an even
    and an odd one (no code structure: the decoders only see LLRs)."""
    from workload.basegraph import custom_base_graph
    rng = np.random.default_rng(77)
    ent = {(0, c): int(rng.integers(0, 384)) for c in range(27)}          # degree 27: columns 0..26
    ent.update({(1, 26): 5, (1, 27): 300})                                 # degree 2
    ent.update({(2, 0): 7, (2, 13): 200, (2, 27): 31, (2, 28): 0})         # degree 4
    ent.update({(3, 1): 90, (3, 2): 2, (3, 3): 383, (3, 28): 64, (3, 29): 1})  # degree 5
    return custom_base_graph("extreme", 4, 30, 26, 4, 0, ent)


@pytest.mark.parametrize("mode", ["f32", "i8", "i16"])
def test_extreme_row_degrees_match_oracle(mode):
    # the sign-history and argmin packing at its limits (edges 0 and 26 of a 27-edge row), the odd last
    # edge, a degree-2 row; Z = 16 (half-warp groups), 32 and 64; an odd block count (a pair without its
    # second block in the paired INT8 kernel)
    from workload.configs import TBSpec, build
    bg = _extreme_degree_graph()
    assert sorted(np.bincount(bg.row).tolist()) == [2, 4, 5, 27]
    specs, widths, punct = [], [], []
    for i, Z in enumerate([16, 32, 32, 32, 64, 64, 64, 32, 16]):
        E = bg.nb * Z
        width = 12 * -(-(E // 2) // (12 * 14))
        specs.append(TBSpec(i, 0, Z, 2, E, 1, 0.9, 0, width))
        widths.append(width)
        punct.append(np.zeros((14, width), bool))
    w = build("extreme", [bg], specs, widths, punct, seed=5, z_set=[16, 32, 64])
    llr = _oracle_llr_for_mode(w, mode)
    want_bits, want_status = odec.decode_workload(w, llr, 5, False, ARITH[mode])
    s = session_for(w, mode, max_iter=5, early_term=False)
    b = s.batch(w.cbs)
    bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
    status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
    s.decode_batch(b, torch.from_numpy(llr.astype(LLR_NP[mode])).cuda(), bits, status)
    assert np.array_equal(to_np_u32(bits), want_bits)
    assert np.array_equal(status.cpu().numpy(), want_status)
    assert s.device_errors() == 0


def _every_degree_graph():
    """26 x 30 base matrix with one row of every degree the decoders accept, 2 .. 27, in a shuffled order, so
    that every leaf of the degree dispatch runs (no code structure: the decoders only see LLRs)."""
    from workload.basegraph import custom_base_graph
    rng = np.random.default_rng(78)
    degrees = rng.permutation(np.arange(2, 28))
    ent = {}
    for r, d in enumerate(degrees):
        for c in rng.choice(30, size=int(d), replace=False):
            ent[(r, int(c))] = int(rng.integers(0, 384))
    return custom_base_graph("every_degree", 26, 30, 4, 26, 0, ent)


def _every_degree_workload(zs, seed):
    from workload.configs import TBSpec, build
    bg = _every_degree_graph()
    assert sorted(np.bincount(bg.row).tolist()) == list(range(2, 28))
    specs, widths, punct = [], [], []
    for i, Z in enumerate(zs):
        E = bg.nb * Z
        width = 12 * -(-(E // 2) // (12 * 14))
        specs.append(TBSpec(i, 0, Z, 2, E, 1, 1.2, 0, width))
        widths.append(width)
        punct.append(np.zeros((14, width), bool))
    return build("every_degree", [bg], specs, widths, punct, seed=seed, z_set=sorted(set(zs)))


@pytest.mark.parametrize("mode", ["f32", "i8", "i16"])
def test_every_row_degree_matches_oracle(mode):
    # every degree from 2 to 27 in one graph, every row decoded; Z = 16 (the single-block INT8 form) and
    # 32/64 (the paired INT8 form), an odd block count
    w = _every_degree_workload([16, 32, 64, 32, 16, 64, 32], seed=6)
    assert all(int(c["Z"]) * 26 <= int(c["E"]) for c in w.cbs)
    llr = _oracle_llr_for_mode(w, mode)
    want_bits, want_status = odec.decode_workload(w, llr, 5, False, ARITH[mode])
    s = session_for(w, mode, max_iter=5, early_term=False)
    b = s.batch(w.cbs)
    bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
    status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
    s.decode_batch(b, torch.from_numpy(llr.astype(LLR_NP[mode])).cuda(), bits, status)
    assert np.array_equal(to_np_u32(bits), want_bits)
    assert np.array_equal(status.cpu().numpy(), want_status)
    assert s.device_errors() == 0


@pytest.mark.parametrize("mode", ["f32", "i8"])
def test_every_row_degree_cluster_matches_oracle(mode):
    # the cluster decoder's copy of the update on the same graph: Z = 64 on 2 CTAs, Z = 128 on 4
    for zs, C in (([64, 64, 64], 2), ([128, 128], 4)):
        w = _every_degree_workload(zs, seed=7 + C)
        llr = _oracle_llr_for_mode(w, mode)
        want_bits, want_status = odec.decode_workload(w, llr, 5, False, ARITH[mode])
        s = session_for(w, mode, max_iter=5, early_term=False)
        b = s.batch(w.cbs)
        bits = torch.zeros(b.info.bits_words, dtype=torch.int32, device="cuda")
        status = torch.zeros(b.n_cb, dtype=torch.int32, device="cuda")
        s.decode_cluster(b, torch.from_numpy(llr.astype(LLR_NP[mode])).cuda(), bits, status, C)
        torch.cuda.synchronize()
        assert np.array_equal(to_np_u32(bits), want_bits), (zs, C)
        assert np.array_equal(status.cpu().numpy(), want_status), (zs, C)
        assert s.device_errors() == 0
