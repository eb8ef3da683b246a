"""Python-side handles for ldpcgb sessions and batches.

``Session`` owns an ``ldpc_session`` (shift tables, workspace, error word) on
the current CUDA device; ``Batch`` owns an ``ldpc_batch`` (validated
descriptors and the decoder's work plan).  Compute methods take torch CUDA
tensors, check their dtype, device and size against the batch, bind the
session to torch's current stream and call the C-ABI.  Nothing here computes
any step of the receive path.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import abi

LLR_TORCH = {"f32": torch.float32, "i8": torch.int8, "i16": torch.int16}
DEFAULT_SAT = {"f32": (0, 0, 0), "i8": (63, 63, 127), "i16": (1023, 1023, 32767)}


def _as_struct_array(arr: np.ndarray, np_dtype: np.dtype) -> np.ndarray:
    a = np.ascontiguousarray(arr)
    if a.dtype.itemsize != np_dtype.itemsize or set(a.dtype.names or ()) - set(np_dtype.names):
        raise TypeError("descriptor array does not match the C layout")
    out = np.zeros(a.shape[0], dtype=np_dtype)
    for name in np_dtype.names:
        out[name] = a[name]
    return out


def _check_tensor(t: torch.Tensor, dtype, min_elems: int, name: str, device) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if t.device.type != "cuda" or (device is not None and t.device.index != device):
        raise ValueError(f"{name}: must live on cuda:{device}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.numel() < min_elems:
        raise ValueError(f"{name}: {t.numel()} elements, the batch needs {min_elems}")
    return t.data_ptr()


class Batch:
    def __init__(self, session: "Session", handle: int, info: abi.BatchInfoC):
        self.session = session
        self.handle = handle
        self.info = info

    def close(self) -> None:
        if self.handle:
            abi.check(abi.load().ldpc_batch_destroy(self.handle), "ldpc_batch_destroy")
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # sizes the caller's buffers must have
    @property
    def n_cb(self) -> int:
        return self.info.n_cb

    @property
    def info_bits(self) -> int:
        return self.info.info_bits

    def plan(self) -> list:
        """The decoder launches of this batch: dicts of block, grid, smem, n_items, global_messages, max_groups."""
        lib = abi.load()
        n = ctypes.c_int32()
        abi.check(lib.ldpc_batch_plan_get(self.handle, None, 0, ctypes.byref(n)), "ldpc_batch_plan_get")
        arr = (abi.LaunchInfoC * max(1, n.value))()
        abi.check(lib.ldpc_batch_plan_get(self.handle, arr, n.value, ctypes.byref(n)), "ldpc_batch_plan_get")
        return [{f: getattr(arr[i], f) for f, _ in abi.LaunchInfoC._fields_} for i in range(n.value)]

    def alloc_outputs(self, device=None) -> dict:
        dev = torch.device("cuda", self.session.device if device is None else device)
        i = self.info
        return dict(
            llr=torch.empty(i.llr_elems, dtype=LLR_TORCH[self.session.mode], device=dev),
            bits=torch.empty(i.bits_words, dtype=torch.int32, device=dev),
            status=torch.empty(i.n_cb, dtype=torch.int32, device=dev),
            d=torch.empty(max(i.n_tb, 1), dtype=torch.uint8, device=dev),
            goodput_bits=torch.empty(max(i.n_slots, 1), dtype=torch.int64, device=dev),
            goodput_sc=torch.empty(max(i.n_slots, 1), dtype=torch.int32, device=dev),
            reward=torch.empty(max(i.n_slots, 1), dtype=torch.float32, device=dev),
        )


class Session:
    """One decoder configuration on one CUDA device."""

    def __init__(self, base_graphs, z_set, mode: str = "f32", max_iter: int = 10, early_term: bool = True,
                 offset_f32: float = 0.5, offset_lsb: int = 1, q_scale: float = 4.0, sat=None,
                 interleave: bool = True, mem_budget: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("ldpcgb needs a CUDA device; there is no CPU path")
        lib = abi.load()
        self.mode = mode
        self.device = torch.cuda.current_device()
        self.n_bg = len(base_graphs)
        self.z_set = [int(z) for z in z_set]
        llr_sat, msg_sat, post_sat = DEFAULT_SAT[mode] if sat is None else sat
        self._keep = []
        bgs = (abi.BaseGraphC * len(base_graphs))()
        for i, g in enumerate(base_graphs):
            row = np.ascontiguousarray(g.row, dtype=np.int16)
            col = np.ascontiguousarray(g.col, dtype=np.int16)
            V = np.ascontiguousarray(g.V, dtype=np.int16)
            self._keep += [row, col, V]
            p16 = ctypes.POINTER(ctypes.c_int16)
            bgs[i] = abi.BaseGraphC(g.mb, g.nb, g.kb, g.mc, g.n_punct_cols, row.size,
                                    row.ctypes.data_as(p16), col.ctypes.data_as(p16), V.ctypes.data_as(p16))
        zs = (ctypes.c_int32 * len(z_set))(*[int(z) for z in z_set])
        desc = abi.SessionDescC(len(base_graphs), bgs, len(z_set), zs, abi.MODES[mode], int(max_iter),
                                int(bool(early_term)), float(offset_f32), int(offset_lsb), float(q_scale),
                                int(llr_sat), int(msg_sat), int(post_sat), int(bool(interleave)),
                                int(mem_budget), None)
        h = ctypes.c_void_p()
        abi.check(lib.ldpc_session_create(ctypes.byref(desc), ctypes.byref(h)), "ldpc_session_create")
        self.handle = h.value
        self._keep = []

    def close(self) -> None:
        if getattr(self, "handle", 0):
            abi.check(abi.load().ldpc_session_destroy(self.handle), "ldpc_session_destroy")
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind_stream(self) -> None:
        s = torch.cuda.current_stream(self.device).cuda_stream
        abi.check(abi.load().ldpc_session_set_stream(self.handle, s), "ldpc_session_set_stream")

    def batch(self, cbs: np.ndarray, tbs: np.ndarray | None = None, slot_N=None) -> Batch:
        lib = abi.load()
        c = _as_struct_array(cbs, abi.CB_NP)
        t = _as_struct_array(tbs, abi.TB_NP) if tbs is not None and len(tbs) else np.zeros(0, abi.TB_NP)
        sn = np.ascontiguousarray(np.zeros(0) if slot_N is None else slot_N, dtype=np.int32)
        h = ctypes.c_void_p()
        abi.check(lib.ldpc_batch_create(self.handle, c.ctypes.data, c.size, t.ctypes.data if t.size else None,
                                        t.size, sn.size, sn.ctypes.data if sn.size else None, ctypes.byref(h)),
                  "ldpc_batch_create")
        info = abi.BatchInfoC()
        abi.check(lib.ldpc_batch_info_get(h.value, ctypes.byref(info)), "ldpc_batch_info_get")
        return Batch(self, h.value, info)

    # ------------------------------------------------------------------ compute
    def puncture_demap(self, b: Batch, sym: torch.Tensor, mask: torch.Tensor, llr: torch.Tensor) -> None:
        i = b.info
        ps = _check_tensor(sym, torch.complex64, i.sym_elems, "sym", self.device)
        pm = _check_tensor(mask, torch.int32, i.mask_words, "mask", self.device)
        pl = _check_tensor(llr, LLR_TORCH[self.mode], i.llr_elems, "llr", self.device)
        self._bind_stream()
        abi.check(abi.load().puncture_demap(self.handle, b.handle, ps, pm, pl), "puncture_demap")

    def decode_batch(self, b: Batch, llr: torch.Tensor, bits: torch.Tensor, status: torch.Tensor) -> None:
        i = b.info
        pl = _check_tensor(llr, LLR_TORCH[self.mode], i.llr_elems, "llr", self.device)
        pb = _check_tensor(bits, torch.int32, i.bits_words, "bits", self.device)
        pst = _check_tensor(status, torch.int32, i.n_cb, "status", self.device)
        self._bind_stream()
        abi.check(abi.load().decode_batch(self.handle, b.handle, pl, pb, pst), "decode_batch")

    def decode_cluster(self, b: Batch, llr: torch.Tensor, bits: torch.Tensor, status: torch.Tensor,
                       cluster_ctas: int = 2) -> None:
        """decode_batch with each code block on a cluster of 2 or 4 CTAs (the latency form; same results)."""
        i = b.info
        pl = _check_tensor(llr, LLR_TORCH[self.mode], i.llr_elems, "llr", self.device)
        pb = _check_tensor(bits, torch.int32, i.bits_words, "bits", self.device)
        pst = _check_tensor(status, torch.int32, i.n_cb, "status", self.device)
        self._bind_stream()
        abi.check(abi.load().ldpc_decode_cluster(self.handle, b.handle, pl, pb, pst, int(cluster_ctas)),
                  "ldpc_decode_cluster")

    def tb_crc_goodput(self, b: Batch, bits: torch.Tensor, d: torch.Tensor, goodput_bits: torch.Tensor,
                       goodput_sc: torch.Tensor, reward: torch.Tensor) -> None:
        i = b.info
        pb = _check_tensor(bits, torch.int32, i.bits_words, "bits", self.device)
        pd = _check_tensor(d, torch.uint8, i.n_tb, "d", self.device)
        pg = _check_tensor(goodput_bits, torch.int64, i.n_slots, "goodput_bits", self.device)
        pgs = _check_tensor(goodput_sc, torch.int32, i.n_slots, "goodput_sc", self.device)
        pr = _check_tensor(reward, torch.float32, i.n_slots, "reward", self.device)
        self._bind_stream()
        abi.check(abi.load().tb_crc_goodput(self.handle, b.handle, pb, pd, pg, pgs, pr), "tb_crc_goodput")

    def run(self, b: Batch, sym: torch.Tensor, mask: torch.Tensor, out: dict) -> dict:
        """The whole path: puncture_demap -> decode_batch -> tb_crc_goodput (if the batch has TBs)."""
        self.puncture_demap(b, sym, mask, out["llr"])
        self.decode_batch(b, out["llr"], out["bits"], out["status"])
        if b.info.n_tb:
            self.tb_crc_goodput(b, out["bits"], out["d"], out["goodput_bits"], out["goodput_sc"], out["reward"])
        return out

    # ------------------------------------------------------------------ planning
    def set_tiles(self, tiles) -> None:
        """tiles: iterable of (bg index, Z, G) -- code blocks per decoder work item."""
        tiles = list(tiles)
        arr = (abi.TileC * max(1, len(tiles)))(*[abi.TileC(int(b), int(z), int(g)) for b, z, g in tiles])
        abi.check(abi.load().ldpc_session_set_tiles(self.handle, arr, len(tiles)), "ldpc_session_set_tiles")

    def set_strategy(self, strategy: str) -> None:
        code = {"mixed": abi.PLAN_MIXED, "per_z": abi.PLAN_PER_Z}[strategy]
        abi.check(abi.load().ldpc_session_set_strategy(self.handle, code), "ldpc_session_set_strategy")

    def load_tiles(self, path: str, base_graphs, tag: str | None = None) -> int:
        """Apply the tiles of an autotuner cache entry (see autotune.py) that name this session's shapes;
        returns how many were applied."""
        from .autotune import tiles_from_cache
        t = [x for x in tiles_from_cache(path, base_graphs, self.mode, tag=tag)
             if x[0] < self.n_bg and x[1] in self.z_set]
        if t:
            self.set_tiles(t)
        return len(t)

    def device_errors(self) -> int:
        v = ctypes.c_uint32()
        abi.check(abi.load().ldpc_device_errors(self.handle, ctypes.byref(v)), "ldpc_device_errors")
        return int(v.value)


class Graph:
    """One whole batch step (demap, decode, CRC/goodput) captured as a CUDA graph on fixed buffers."""

    def __init__(self, session: Session, b: Batch, sym: torch.Tensor, mask: torch.Tensor, out: dict):
        i = b.info
        ptrs = [
            _check_tensor(sym, torch.complex64, i.sym_elems, "sym", session.device),
            _check_tensor(mask, torch.int32, i.mask_words, "mask", session.device),
            _check_tensor(out["llr"], LLR_TORCH[session.mode], i.llr_elems, "llr", session.device),
            _check_tensor(out["bits"], torch.int32, i.bits_words, "bits", session.device),
            _check_tensor(out["status"], torch.int32, i.n_cb, "status", session.device),
            _check_tensor(out["d"], torch.uint8, i.n_tb, "d", session.device),
            _check_tensor(out["goodput_bits"], torch.int64, i.n_slots, "goodput_bits", session.device),
            _check_tensor(out["goodput_sc"], torch.int32, i.n_slots, "goodput_sc", session.device),
            _check_tensor(out["reward"], torch.float32, i.n_slots, "reward", session.device),
        ]
        self._keep = (session, b, sym, mask, out)
        h = ctypes.c_void_p()
        abi.check(abi.load().ldpc_graph_create(session.handle, b.handle, *ptrs, ctypes.byref(h)), "ldpc_graph_create")
        self.handle = h.value
        self.device = session.device

    def launch(self) -> None:
        s = torch.cuda.current_stream(self.device).cuda_stream
        abi.check(abi.load().ldpc_graph_launch(self.handle, s), "ldpc_graph_launch")

    def close(self) -> None:
        if getattr(self, "handle", 0):
            abi.check(abi.load().ldpc_graph_destroy(self.handle), "ldpc_graph_destroy")
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching decode service on a session (see the serving section of ldpcgb.h).

    host_pool / result_pool: pinned CPU tensors (``pin_memory()``) holding the
    requests' symbols and masks, and receiving decoded bits.  Requests are
    numpy arrays of ``abi.SERVE_TB_NP``.  ``cb_crc``: accept TBs whose code
    blocks carry their own CRC (the loop runs its CRC-exit variant).
    ``paired``: how an INT8 service decodes a request's code blocks -- ``"auto"``
    (paired, two blocks per thread group, once more than ``pair_threshold``
    work items would be in flight -- 0: two per loop thread block -- and until
    they fall to ``pair_release`` -- 0: one per loop thread block; single
    otherwise), ``True`` (always paired where the shape allows) or ``False``
    (always single).  ``codebook``: ``(bitmaps, prb)``, the URLLC puncturing codebook that requests
    with ``pattern >= 0`` name (``bitmaps``: uint32 [entries][7][ceil(prb / 32)], copied at start).
    """

    def __init__(self, session: Session, host_pool: torch.Tensor, result_pool: torch.Tensor | None = None,
                 arena_bytes: int = 8 << 30, max_inflight: int = 4096, idle_timeout_us: int = 200000,
                 loops_per_sm: int = 1, cb_crc: bool = False, paired: bool | str = "auto",
                 pair_threshold: int = 0, pair_release: int = 0, codebook: np.ndarray | None = None):
        for t, name in ((host_pool, "host_pool"), (result_pool, "result_pool")):
            if t is not None and not (t.device.type == "cpu" and t.is_pinned() and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous pinned CPU tensor")
        self._keep = (session, host_pool, result_pool)
        if paired not in ("auto", True, False):
            raise ValueError("paired must be 'auto', True or False")
        form = 0 if paired == "auto" else (abi.SERVE_PAIRED if paired is True else abi.SERVE_UNPAIRED)
        book_n = book_prb = 0
        book_ptr = None
        if codebook is not None:
            book, book_prb = codebook
            book = np.ascontiguousarray(book, dtype=np.uint32)
            if book.ndim != 3 or book.shape[1] != 7 or book.shape[2] != -(-int(book_prb) // 32):
                raise ValueError("codebook bitmaps must be [entries][7][ceil(prb / 32)] uint32")
            book_n, book_ptr = book.shape[0], book.ctypes.data
        d = abi.ServeDescC(int(arena_bytes), int(max_inflight), int(idle_timeout_us), host_pool.data_ptr(),
                           host_pool.numel() * host_pool.element_size(),
                           result_pool.data_ptr() if result_pool is not None else None,
                           result_pool.numel() * result_pool.element_size() if result_pool is not None else 0,
                           int(loops_per_sm), (abi.SERVE_CB_CRC if cb_crc else 0) | form, int(pair_threshold),
                           int(pair_release), int(book_n), int(book_prb), book_ptr)
        h = ctypes.c_void_p()
        abi.check(abi.load().ldpc_serve_start(session.handle, ctypes.byref(d), ctypes.byref(h)), "ldpc_serve_start")
        self.handle = h.value

    def submit(self, tbs: np.ndarray) -> int:
        a = np.ascontiguousarray(tbs, dtype=abi.SERVE_TB_NP)
        n = ctypes.c_int32()
        abi.check(abi.load().ldpc_serve_submit(self.handle, a.ctypes.data, a.size, ctypes.byref(n)),
                  "ldpc_serve_submit")
        return n.value

    def poll(self, cap: int = 4096) -> np.ndarray:
        out = np.zeros(cap, dtype=abi.SERVE_DONE_NP)
        n = ctypes.c_int32()
        abi.check(abi.load().ldpc_serve_poll(self.handle, out.ctypes.data, cap, ctypes.byref(n)), "ldpc_serve_poll")
        return out[:n.value]

    def replay(self, tbs: np.ndarray, arrival_ns: np.ndarray, timeout_ms: int = 10000) -> np.ndarray:
        a = np.ascontiguousarray(tbs, dtype=abi.SERVE_TB_NP)
        t = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        out = np.empty(a.size, dtype=abi.SERVE_DONE_NP)
        out.view(np.uint8)[:] = 0  # every page touched before the timed loop writes it
        abi.check(abi.load().ldpc_serve_replay(self.handle, a.ctypes.data, t.ctypes.data, a.size, out.ctypes.data,
                                               int(timeout_ms)), "ldpc_serve_replay")
        return out

    def stats(self) -> dict:
        """Counters since start (requests, items admitted single / paired, loop launches) and, for the last
        replay, its host loop's longest pass (ns, and when it began), passes longer than 1 ms, and the
        replaying thread's context switches and page faults."""
        out = (ctypes.c_int64 * 11)()
        abi.check(abi.load().ldpc_serve_stats(self.handle, ctypes.cast(out, ctypes.c_void_p), 11), "ldpc_serve_stats")
        return {"requests": out[0], "items_single": out[1], "items_paired": out[2], "launches": out[3],
                "replay_longest_pass_ns": out[4], "replay_passes_over_1ms": out[5],
                "replay_longest_pass_at_ns": out[6], "replay_involuntary_switches": out[7],
                "replay_voluntary_switches": out[8], "replay_minor_faults": out[9], "replay_major_faults": out[10]}

    def stop(self) -> None:
        if getattr(self, "handle", 0):
            abi.check(abi.load().ldpc_serve_stop(self.handle), "ldpc_serve_stop")
            self.handle = 0

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
