"""ctypes binding of the ldpcgb C-ABI (``include/ldpcgb.h``).

Argument marshalling only: every step of the receive path runs in the CUDA
kernels behind ``libldpcgb.so``.  PyTorch supplies device memory and the
current stream; buffers are passed as raw device pointers.  There is no CPU
fallback: if the library is missing or was built for another GPU, the calls
raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libldpcgb.so")
# LDPCGB_CHECKED=1: the build with device index checks (see ldpc_check_log), built and loaded instead
LIB_PATH_CHECKED = os.path.join(HERE, "libldpcgb_checked.so")

LDPC_F32, LDPC_I8, LDPC_I16 = 0, 1, 2
MODES = {"f32": LDPC_F32, "i8": LDPC_I8, "i16": LDPC_I16}
ERRORS = {-1: "LDPC_EINVAL", -2: "LDPC_ENOMEM", -3: "LDPC_ECUDA", -4: "LDPC_ETIMEOUT", -5: "LDPC_EBUSY"}

EXPORTED = [
    "ldpc_session_create", "ldpc_session_destroy", "ldpc_session_set_stream",
    "ldpc_batch_create", "ldpc_batch_destroy", "ldpc_batch_info_get",
    "puncture_demap", "decode_batch", "ldpc_decode_cluster", "tb_crc_goodput",
    "ldpc_device_errors", "ldpc_check_log", "ldpc_last_error", "ldpc_version", "decode_uniform_noalloc",
    "decode_uniform_noalloc_errors", "decode_uniform_noalloc_wait_check",
    "ldpc_session_set_tiles", "ldpc_session_set_strategy", "ldpc_batch_plan_get",
    "ldpc_graph_create", "ldpc_graph_launch", "ldpc_graph_destroy",
    "ldpc_serve_start", "ldpc_serve_submit", "ldpc_serve_poll", "ldpc_serve_replay", "ldpc_serve_stats",
    "ldpc_serve_stop",
    "ldpc_puncture_alloc", "ldpc_feasibility_enforce", "ldpc_sc_mask", "ldpc_rt_odu_codebook",
]
POLICY_RP, POLICY_SEF = 0, 1
PLAN_MIXED, PLAN_PER_Z = 0, 1


class BaseGraphC(ctypes.Structure):
    _fields_ = [("mb", ctypes.c_int32), ("nb", ctypes.c_int32), ("kb", ctypes.c_int32), ("mc", ctypes.c_int32),
                ("n_punct_cols", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("row", ctypes.POINTER(ctypes.c_int16)), ("col", ctypes.POINTER(ctypes.c_int16)),
                ("V", ctypes.POINTER(ctypes.c_int16))]


class SessionDescC(ctypes.Structure):
    _fields_ = [("n_bg", ctypes.c_int32), ("bgs", ctypes.POINTER(BaseGraphC)),
                ("n_z", ctypes.c_int32), ("z_set", ctypes.POINTER(ctypes.c_int32)),
                ("mode", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("early_term", ctypes.c_int32),
                ("offset_f32", ctypes.c_float), ("offset_lsb", ctypes.c_int32), ("q_scale", ctypes.c_float),
                ("llr_sat", ctypes.c_int32), ("msg_sat", ctypes.c_int32), ("post_sat", ctypes.c_int32),
                ("interleave", ctypes.c_int32), ("device_mem_budget", ctypes.c_uint64),
                ("cuda_stream", ctypes.c_void_p)]


class CbDescC(ctypes.Structure):
    _fields_ = [("bg", ctypes.c_int32), ("Z", ctypes.c_int32), ("Qm", ctypes.c_int32), ("E", ctypes.c_int32),
                ("re_offset", ctypes.c_int64), ("mask_word_offset", ctypes.c_int64),
                ("llr_offset", ctypes.c_int64), ("bits_word_offset", ctypes.c_int64),
                ("inv_sigma2", ctypes.c_float), ("flags", ctypes.c_int32)]


CB_FLAG_CRC24B = 1  # the code block's last 24 information bits are a CRC (0x800063) of the others
CB_RV_SHIFT = 1     # flags bits 1-2: the redundancy version sent (LDPC_CB_RV)


class TbDescC(ctypes.Structure):
    _fields_ = [("first_cb", ctypes.c_int32), ("n_cb", ctypes.c_int32), ("n_sc", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("payload_bits", ctypes.c_int32)]


class TileC(ctypes.Structure):
    _fields_ = [("bg", ctypes.c_int32), ("Z", ctypes.c_int32), ("G", ctypes.c_int32)]


class LaunchInfoC(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("grid", ctypes.c_int32), ("smem", ctypes.c_int32),
                ("n_items", ctypes.c_int32), ("global_messages", ctypes.c_int32), ("max_groups", ctypes.c_int32)]


class ServeDescC(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_int32),
                ("idle_timeout_us", ctypes.c_int32), ("host_pool", ctypes.c_void_p),
                ("host_pool_bytes", ctypes.c_uint64), ("result_pool", ctypes.c_void_p),
                ("result_pool_bytes", ctypes.c_uint64), ("loops_per_sm", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("pair_threshold", ctypes.c_int32), ("pair_release", ctypes.c_int32),
                ("codebook_n", ctypes.c_int32), ("codebook_prb", ctypes.c_int32), ("codebook", ctypes.c_void_p)]


SERVE_CB_CRC = 1  # ldpc_serve_desc.flags: accept TBs with code-block CRCs
SERVE_UNPAIRED = 2  # ldpc_serve_desc.flags: INT8 requests always in the single form
SERVE_PAIRED = 4  # ldpc_serve_desc.flags: INT8 requests always in the paired form (where the shape allows)


class ServeTbC(ctypes.Structure):
    _fields_ = [("bg", ctypes.c_int32), ("Z", ctypes.c_int32), ("Qm", ctypes.c_int32), ("E", ctypes.c_int32),
                ("n_cb", ctypes.c_int32), ("n_sc", ctypes.c_int32), ("payload_bits", ctypes.c_int32),
                ("inv_sigma2", ctypes.c_float), ("rv", ctypes.c_int32), ("pattern", ctypes.c_int32),
                ("sym_offset", ctypes.c_int64), ("mask_offset", ctypes.c_int64),
                ("result_offset", ctypes.c_int64), ("tag", ctypes.c_uint64), ("grid_sc", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServeDoneC(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("d", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("all_syndrome_ok", ctypes.c_int32), ("status", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_int64), ("t_complete_ns", ctypes.c_int64),
                ("t_device_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64)]


class BatchInfoC(ctypes.Structure):
    _fields_ = [("sym_elems", ctypes.c_int64), ("mask_words", ctypes.c_int64), ("llr_elems", ctypes.c_int64),
                ("bits_words", ctypes.c_int64), ("n_cb", ctypes.c_int32), ("n_tb", ctypes.c_int32),
                ("n_slots", ctypes.c_int32), ("n_items", ctypes.c_int32), ("info_bits", ctypes.c_int64)]


def _np_dtype(struct) -> np.dtype:
    """NumPy structured dtype with the exact field offsets of a ctypes struct."""
    conv = {ctypes.c_int32: "<i4", ctypes.c_int64: "<i8", ctypes.c_float: "<f4"}
    names, formats, offsets = [], [], []
    for name, ct in struct._fields_:
        names.append(name)
        formats.append(conv[ct])
        offsets.append(getattr(struct, name).offset)
    return np.dtype({"names": names, "formats": formats, "offsets": offsets, "itemsize": ctypes.sizeof(struct)})


CB_NP = _np_dtype(CbDescC)
TB_NP = _np_dtype(TbDescC)


def _np_dtype_any(struct) -> np.dtype:
    conv = {ctypes.c_int32: "<i4", ctypes.c_int64: "<i8", ctypes.c_float: "<f4", ctypes.c_uint64: "<u8"}
    names = [n for n, _ in struct._fields_]
    return np.dtype({"names": names, "formats": [conv[t] for _, t in struct._fields_],
                     "offsets": [getattr(struct, n).offset for n in names], "itemsize": ctypes.sizeof(struct)})


SERVE_TB_NP = _np_dtype_any(ServeTbC)
SERVE_DONE_NP = _np_dtype_any(ServeDoneC)

_lib = None


class LdpcError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libldpcgb.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or (LIB_PATH_CHECKED if os.environ.get("LDPCGB_CHECKED") == "1" else LIB_PATH)
    if not os.path.exists(p):
        raise OSError(f"libldpcgb.so not found at {p}; run paper_2506_00167_gb300.build.build() first")
    lib = ctypes.CDLL(p)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.ldpc_session_create.argtypes = [ctypes.POINTER(SessionDescC), ctypes.POINTER(vp)]
    lib.ldpc_session_destroy.argtypes = [vp]
    lib.ldpc_session_set_stream.argtypes = [vp, vp]
    lib.ldpc_batch_create.argtypes = [vp, vp, i32, vp, i32, i32, vp, ctypes.POINTER(vp)]
    lib.ldpc_batch_destroy.argtypes = [vp]
    lib.ldpc_batch_info_get.argtypes = [vp, ctypes.POINTER(BatchInfoC)]
    lib.puncture_demap.argtypes = [vp, vp, vp, vp, vp]
    lib.decode_batch.argtypes = [vp, vp, vp, vp, vp]
    lib.ldpc_decode_cluster.argtypes = [vp, vp, vp, vp, vp, i32]
    lib.tb_crc_goodput.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.ldpc_device_errors.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
    lib.ldpc_check_log.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
    lib.decode_uniform_noalloc.argtypes = [ctypes.POINTER(BaseGraphC), i32, i32, i32, i32, i32, i32,
                                           ctypes.c_float, i32, i32, i32, vp, vp, vp, vp]
    lib.decode_uniform_noalloc_errors.argtypes = [ctypes.POINTER(ctypes.c_uint32), vp]
    lib.decode_uniform_noalloc_wait_check.argtypes = [i32, vp]
    lib.ldpc_session_set_tiles.argtypes = [vp, ctypes.POINTER(TileC), i32]
    lib.ldpc_session_set_strategy.argtypes = [vp, i32]
    lib.ldpc_batch_plan_get.argtypes = [vp, ctypes.POINTER(LaunchInfoC), i32, ctypes.POINTER(i32)]
    lib.ldpc_graph_create.argtypes = [vp] * 11 + [ctypes.POINTER(vp)]
    lib.ldpc_graph_launch.argtypes = [vp, vp]
    lib.ldpc_graph_destroy.argtypes = [vp]
    lib.ldpc_serve_start.argtypes = [vp, ctypes.POINTER(ServeDescC), ctypes.POINTER(vp)]
    lib.ldpc_serve_submit.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
    lib.ldpc_serve_poll.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
    lib.ldpc_serve_replay.argtypes = [vp, vp, vp, i32, vp, i32]
    lib.ldpc_serve_stats.argtypes = [vp, vp, i32]
    lib.ldpc_serve_stop.argtypes = [vp]
    lib.ldpc_last_error.restype = ctypes.c_char_p
    lib.ldpc_version.restype = ctypes.c_char_p
    for name in EXPORTED:
        f = getattr(lib, name)
        if f.restype is None or f.restype is ctypes.c_int:
            f.restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def check(rc: int, where: str) -> None:
    if rc != 0:
        msg = load().ldpc_last_error().decode(errors="replace")
        raise LdpcError(rc, where, msg)
