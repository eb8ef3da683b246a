"""The cluster decoder (each code block on 2 or 4 CTAs, posteriors replicated): bit-identical to decode_batch in
every mode, INT8 bit-exact against the oracle's integer decoder, refusals for shapes it cannot split."""
import numpy as np
import pytest
import torch

from oracle import decoder as odec
from oracle import demap as odemap
from paper_2506_00167_gb300 import LdpcError
from workload import large_fp32, mixed
from workload.configs import subset

from gpu_helpers import LLR_NP, batch_for, device_inputs, session_for

pytestmark = pytest.mark.gpu


def _mixed_z(min_z):
    w = mixed(n_slots=6, ues_per_slot=4, max_cb=3)
    keep = [t for t in range(w.n_tb) if int(w.cbs[int(w.tbs[t]["first_cb"])]["Z"]) % min_z == 0]
    return subset(w, keep)


@pytest.fixture(scope="module")
def wls():
    return {"large": large_fp32(n_cw=8, snr_points=(6, 8, 10, 12)), "mixed64": _mixed_z(64), "mixed128": _mixed_z(128)}


@pytest.mark.parametrize("mode", ["f32", "i16", "i8"])
@pytest.mark.parametrize("name,C", [("large", 2), ("large", 4), ("mixed64", 2), ("mixed128", 4)])
def test_cluster_decode_equals_decode_batch(wls, name, C, mode):
    w = wls[name]
    s = session_for(w, mode)
    b = batch_for(s, w)
    sym, mask = device_inputs(w)
    ref = s.run(b, sym, mask, b.alloc_outputs())
    bits = torch.full_like(ref["bits"], -1)
    status = torch.full_like(ref["status"], -1)
    for _ in range(2):  # the first call builds the cluster plan, the second reuses it
        s.decode_cluster(b, ref["llr"], bits, status, C)
        torch.cuda.synchronize()
        assert torch.equal(bits, ref["bits"])
        assert torch.equal(status, ref["status"])
    assert s.device_errors() == 0


def test_cluster_int8_is_bit_exact_against_the_oracle(wls):
    w = wls["large"]
    llr = odemap.quantise(odemap.demap_workload(w), 4.0, 63).astype(np.int8)
    want_bits, want_status = odec.decode_workload(w, llr, 10, True, odec.INT8)
    s = session_for(w, "i8")
    b = batch_for(s, w)
    out = b.alloc_outputs()
    s.decode_cluster(b, torch.from_numpy(llr).cuda(), out["bits"], out["status"], 4)
    torch.cuda.synchronize()
    assert np.array_equal(out["bits"].cpu().numpy().view(np.uint32), want_bits)
    assert np.array_equal(out["status"].cpu().numpy(), want_status)


def test_cluster_refuses_what_it_cannot_split(wls):
    w = _mixed_z(32)
    s = session_for(w, "f32")
    b = batch_for(s, w)
    out = b.alloc_outputs()
    llr = torch.zeros(b.info.llr_elems, dtype=torch.float32, device="cuda")
    if np.any(w.cbs["Z"] % 128):
        with pytest.raises(LdpcError, match="does not split"):
            s.decode_cluster(b, llr, out["bits"], out["status"], 4)
    with pytest.raises(LdpcError, match="2 or 4"):
        s.decode_cluster(b, llr, out["bits"], out["status"], 3)
