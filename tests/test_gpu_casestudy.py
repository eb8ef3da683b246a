"""The case-study link path: policy -> SC masks -> transmit chain -> GPU receive path -> d_e, reward."""
import numpy as np
import pytest
import torch

from oracle import path as opath
from oracle import policy as P
from paper_2506_00167_gb300 import policy as G
from workload.policy import N_SC, case_study, schedules

from gpu_helpers import device_inputs, session_for

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("policy", ["rp", "sef"])
def test_policy_masks_drive_the_receive_path(policy):
    T = 12
    alloc, demand = schedules(T, seed=31)
    # masks on the GPU equal the oracle's
    pm, st = G.puncture_alloc(torch.from_numpy(alloc.astype(np.int32)).cuda(),
                              torch.from_numpy(demand.astype(np.int32)).cuda(), policy)
    words = (N_SC + 31) // 32
    gm = G.sc_mask(torch.from_numpy(alloc.astype(np.int32)).cuda(), pm, words).cpu().numpy().astype("<u4")
    bits = np.unpackbits(gm.view(np.uint8), bitorder="little").reshape(T, 14, -1)[:, :, :N_SC].astype(bool)
    masks = [P.sc_mask(alloc[t], P.allocate(alloc[t], demand[t], policy)) for t in range(T)]
    assert int(st.sum()) == 0
    assert all(np.array_equal(bits[t], masks[t]) for t in range(T))
    # the receive path on TTIs built from the oracle's masks
    w = case_study(alloc, masks, seed=32)
    ref = opath.run(w, "f64", 10, True)
    s = session_for(w, "f32")
    b = s.batch(w.cbs, w.tbs, w.slot_N)
    sym, mask = device_inputs(w)
    out = s.run(b, sym, mask, b.alloc_outputs())
    d = out["d"].cpu().numpy()
    assert np.mean(d == ref["d"]) >= 0.97
    # eq. 2 per TTI from the GPU's own d_e
    r = out["reward"].cpu().numpy()
    want = np.array([-(alloc[t] * (1 - d[t * 10:(t + 1) * 10])).sum() / 780.0 for t in range(T)], dtype=np.float32)
    assert np.allclose(r, want, rtol=0, atol=1e-6)
