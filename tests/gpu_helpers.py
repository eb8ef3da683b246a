"""Shared helpers for the GPU tests: move a workload to the device, build sessions."""
import numpy as np
import torch

from paper_2506_00167_gb300 import Session

SAT = {"f32": None, "i8": (63, 63, 127), "i16": (1023, 1023, 32767)}


def session_for(w, mode, max_iter=None, early_term=None, **kw):
    mi = w.meta.get("max_iter", 10) if max_iter is None else max_iter
    et = w.meta.get("early_term", 1) if early_term is None else early_term
    return Session(w.bgs, w.z_set, mode=mode, max_iter=mi, early_term=bool(et), sat=SAT[mode], **kw)


def device_inputs(w, dev="cuda"):
    sym = torch.from_numpy(np.ascontiguousarray(w.sym, dtype=np.complex64)).to(dev)
    mask = torch.from_numpy(np.ascontiguousarray(w.mask).view(np.int32)).to(dev)
    return sym, mask


def batch_for(s, w, with_tbs=True):
    if with_tbs:
        return s.batch(w.cbs, w.tbs, w.slot_N)
    return s.batch(w.cbs)


def to_np_u32(t):
    return t.cpu().numpy().view(np.uint32)


LLR_NP = {"f32": np.float32, "i8": np.int8, "i16": np.int16}
