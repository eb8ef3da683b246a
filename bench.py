"""Benchmark: decoded information Gbit/s of the punctured-eMBB receive path on GB300.

One step = one pass of the whole path over one batch: puncture flushing +
max-log demap -> layered offset-min-sum decode -> TB CRC-24, goodput and
reward.  Default workload: 4096 BG1-shaped code blocks, Z = 384 (K = 8448),
rate 1/2, 16-QAM, Es/N0 cycling 6..12 dB, URLLC preempting 1-3 mini-slots on
4-12 PRBs per slot, 10 iterations with early termination, float32.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun each rank decodes its own replica of the
workload (independent code blocks: no collective on the data path) and the
value is all ranks' decoded bits over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "decoded info Gbit/s + % HBM roofline; served p99 slot latency vs 125 µs, INT8 vs FP32"
ALU_OPS_PER_EDGE = 8   # minimal ALU-pipe lane-ops per lifted edge update: R select + sign (2), min1/min2 (3),
                       # sign parity (1), new magnitude select (1), new sign (1)
ALU_LANES_PER_SM = 64  # ALU pipe (min/max/compare/select/logic): 64 lanes per clock per SM
SAT = {"f32": None, "i8": (63, 63, 127), "i16": (1023, 1023, 32767)}


# ----------------------------------------------------------------------------- CPU oracle leg
def _oracle_chunk(args):
    """Worker: run the oracle path on a sub-workload; returns (info bits, failed TBs)."""
    w, mode, max_iter, et = args
    from oracle import path as opath
    out = opath.run(w, mode, max_iter, et)
    return int(sum(w.bgs[int(c["bg"])].kb * int(c["Z"]) for c in w.cbs)), int((out["d"] == 0).sum())


def make_workload(name: str, rank: int = 0, n: int | None = None, cb_crc: bool = False):
    from workload import large_fp32, mixed, tiny_fp32
    if name == "large":
        return large_fp32(n_cw=n or 4096, seed=2 + 1000 * rank)
    if name == "mixed":
        return mixed(n_slots=n or 512, seed=3 + 1000 * rank, cb_crc=cb_crc)
    if name == "tiny":
        return tiny_fp32(seed=1000 * rank)
    raise ValueError(name)


def reduce_over_ranks(ms: float, units: int, world: int, device=None):
    """(slowest rank's time, all ranks' units): the timing contract across replicas."""
    if world == 1:
        return ms, units
    import torch
    import torch.distributed as dist
    t_ms = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    t_u = torch.tensor([int(units)], dtype=torch.int64, device=device)
    dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    dist.all_reduce(t_u, op=dist.ReduceOp.SUM)
    return float(t_ms.item()), int(t_u.item())


def oracle_sample(w, n_tb: int, n_chunks: int):
    from workload.configs import subset
    idx = np.arange(min(n_tb, w.n_tb))
    return [subset(w, part) for part in np.array_split(idx, n_chunks) if part.size]


def time_oracle(pool, chunks, mode, max_iter, et):
    t = time.perf_counter()
    res = pool.map(_oracle_chunk, [(c, mode, max_iter, et) for c in chunks])
    dt = time.perf_counter() - t
    return sum(r[0] for r in res), dt


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        # raw samples: a per-process file in BENCH_CLOCKS_DIR (default: the system temp directory)
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu_id], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = [ln.split(",") for ln in open(self.path) if ln.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- helpers
def edge_updates(w, status: np.ndarray) -> int:
    """Lifted edge updates the decoder performed: sum over blocks of iterations x edges in m_eff rows x Z."""
    total = 0
    cache = {}
    for i, c in enumerate(w.cbs):
        bg, Z, t0, m_eff, n_eff = w.cb_geometry(i)
        key = (int(c["bg"]), m_eff)
        if key not in cache:
            cache[key] = int(np.sum(bg.row < m_eff))
        total += int(status[i] & 0xFFFF) * cache[key] * Z
    return total


def hbm_bytes(w, mode: str) -> dict:
    """Algorithmic DRAM bytes per step for each kernel (read + write)."""
    esz = {"f32": 4, "i8": 1, "i16": 2}[mode]
    sym = w.sym.size * 8
    mask = w.mask.size * 4
    llr = w.llr_len * esz
    bits = w.bits_words * 4
    status = w.n_cb * 4
    return {"demap": sym + mask + llr, "decode": llr + bits + status,
            "crc": bits + w.n_tb * 1 + w.n_slots * 16}


def peak_alu_gops(num_sms: int, mhz: float) -> float:
    """ALU-pipe lane-ops per second: SMs x 64 lanes x clock."""
    return num_sms * ALU_LANES_PER_SM * mhz * 1e6 / 1e9


def decoder_traffic(mode: str, n_cb: int, config: str):
    """DRAM bytes per decode launch from the committed ncu capture, or None if the decoder changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "decode_traffic.json")
    if config != "large" or not os.path.exists(path):
        return None
    rec = json.load(open(path))
    src = b"".join(open(os.path.join(ROOT, "paper_2506_00167_gb300", "csrc", f), "rb").read()
                   for f in ("decode.cu", "decode_core.cuh", "internal.cuh"))
    if hashlib.sha256(src).hexdigest()[:16] != rec.get("decoder_source_sha256_16"):
        return None
    m = rec["modes"].get(mode)
    return None if m is None else m["bytes_per_launch_full"] * n_cb / m["scaled_to"]


TILE_CACHE = os.path.join(ROOT, "results", "autotune_tiles.json")


def apply_tiles(s, w, mode: str, how: str, world: int = 1):
    """Work-item tiles for the session: 'auto' = the autotuner's cache for this GPU and mode (tuned now, on
    the workload's shapes, when the cache has no entry and the run has one rank), 'default' = built-in
    tiles, else a cache path."""
    if how == "default":
        return {"source": "built-in default"}
    path = TILE_CACHE if how == "auto" else how
    tag = w.meta.get("name")
    n = s.load_tiles(path, w.bgs, tag=tag)
    tuned_now = False
    if n == 0 and how == "auto" and world == 1:
        from paper_2506_00167_gb300.autotune import autotune_batch
        autotune_batch(w.bgs, w.z_set, w.cbs, mode=mode, max_iter=3, reps=3, cache_path=path, tag=tag)
        n = s.load_tiles(path, w.bgs, tag=tag)
        tuned_now = True
    if n == 0:
        return {"source": "built-in default (no autotuner entry for this GPU)"}
    return {"source": "autotuner cache " + os.path.relpath(path, ROOT) + (" (tuned in this run)" if tuned_now else ""),
            "shapes": n}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured", float(d.get("sm_max_mhz", 2070.0))
    return 6800.0, "fallback", 2070.0


def workload_desc(args) -> str:
    """The workload named in both arms' JSON lines."""
    return {"large": "4096 x BG1-shaped Z=384 K=8448 R=1/2 16-QAM, Es/N0 6-12 dB, <=10 iter + ET",
            "mixed": "512 slots x 8 UEs mixed BG/Z/R/Qm" + (", CRC-24B per code block" if args.cb_crc else ""),
            "tiny": "8x16 Z=16 QPSK"}[args.config]


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, world, rank):
    if rank != 0:
        return
    w = make_workload(args.config, cb_crc=args.cb_crc)
    mi, et = w.meta["max_iter"], bool(w.meta["early_term"])
    mode = "f64"
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    per_step_tb = args.ref_tb
    with ctx.Pool(cores) as pool:
        chunks = oracle_sample(w, per_step_tb, cores)
        for _ in range(args.warmup):
            time_oracle(pool, chunks, mode, mi, et)
        bits = 0
        dt = 0.0
        for _ in range(args.steps):
            b, t = time_oracle(pool, chunks, mode, mi, et)
            bits += b
            dt += t
    v = bits / dt / 1e9
    sample = f"first {per_step_tb} TBs of the {args.config} workload per step, float64 oracle, {cores} processes"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gbit/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(args), "cb_crc": bool(args.cb_crc)},
            "cpu_baseline": {"value": v, "unit": "Gbit/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- precision sweep
def _oracle_errors(args):
    """Worker: per-block errors of the float64 oracle on one noisy sub-batch."""
    w, mi, et = args
    from oracle import path as opath
    out = opath.run(w, "f64", mi, et)
    return opath.block_errors(w, out["words"])


def run_precision_sweep(args):
    """BLER per Es/N0 point: GPU float32 / INT8 / INT16 against the float64 oracle, 95 % Wilson intervals.

    A pool of noiseless code blocks (URLLC masks included) is encoded once;
    every batch draws fresh seeded AWGN for the whole pool.  The GPU decodes
    args.sweep_n code blocks per point in all three modes; the oracle decodes
    the first args.sweep_oracle_n of them.  ``--config large``: the large
    workload's shape, points in absolute Es/N0.  ``--config mixed``: the mixed
    workload's shapes (BG, Z, R, Qm per TB), each code block at its shape's
    operating point + the point's offset.
    """
    import torch
    from oracle.stats import wilson
    from paper_2506_00167_gb300 import Session
    from workload import large_fp32, mixed
    from workload.configs import es_n0_sigma2, operating_point_db, subset
    from workload.rng import np_stream

    cores = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(cores)
    torch.cuda.set_device(0)
    is_mixed = args.config == "mixed"
    if is_mixed:
        w0 = mixed(n_slots=args.sweep_pool, noiseless=True, seed=41)
        K = np.array([w0.bgs[int(c["bg"])].kb * int(c["Z"]) for c in w0.cbs], np.float64)
        op = np.array([operating_point_db(k / int(c["E"]), int(c["Qm"])) for k, c in zip(K, w0.cbs)])
        points = [float(v) for v in np.arange(args.sweep_lo, args.sweep_lo + 0.5 * 10, 0.5)]
    else:
        w0 = large_fp32(n_cw=args.sweep_pool, noiseless=True, seed=40)
        op = np.zeros(w0.n_cb)
        points = [float(v) for v in np.arange(args.sweep_lo, args.sweep_lo + 0.5 * 10, 0.5)]
    n_pool = w0.n_cb
    mi, et = w0.meta["max_iter"], bool(w0.meta["early_term"])
    x = w0.sym.astype(np.complex128)
    n_re = (w0.cbs["E"] // w0.cbs["Qm"]).astype(np.int64)
    info = torch.from_numpy(w0.info_words.view(np.int32)).cuda()
    words_per_cb = np.array([w0.bgs[int(c["bg"])].kb * int(c["Z"]) // 32 for c in w0.cbs], np.int64)
    word_cb = torch.from_numpy(np.repeat(np.arange(n_pool), words_per_cb)).cuda()
    assert np.array_equal(w0.cbs["bits_word_offset"], np.concatenate([[0], np.cumsum(words_per_cb)[:-1]]))
    mask = torch.from_numpy(w0.mask.view(np.int32)).cuda()
    sess = {m: Session(w0.bgs, w0.z_set, mode=m, max_iter=mi, early_term=et, sat=SAT[m]) for m in ("f32", "i8", "i16")}
    rows = []
    t_start = time.perf_counter()
    for pi, pt in enumerate(points):
        s2_cb = es_n0_sigma2(op + pt)
        s2_re = np.repeat(s2_cb, n_re)
        cbs = w0.cbs.copy()
        cbs["inv_sigma2"] = (1.0 / s2_cb).astype(np.float32)
        batches = {m: sess[m].batch(cbs) for m in sess}
        outs = {m: batches[m].alloc_outputs() for m in sess}
        err = {m: 0 for m in sess}
        iters = {m: 0 for m in sess}
        same = {m: [] for m in sess}  # per-block errors on the blocks the oracle also decodes (same noise)
        n_done = 0
        rng = np_stream(40 + is_mixed, 7, pi)
        oracle_jobs = []
        while n_done < args.sweep_n:
            noise = rng.standard_normal((2, x.size))
            y = (x + np.sqrt(s2_re / 2.0) * (noise[0] + 1j * noise[1])).astype(np.complex64)
            sym = torch.from_numpy(y).cuda()
            for m in sess:
                s, b, o = sess[m], batches[m], outs[m]
                s.puncture_demap(b, sym, mask, o["llr"])
                s.decode_batch(b, o["llr"], o["bits"], o["status"])
                bad_w = (o["bits"] != info).to(torch.int32)
                per_cb = torch.zeros(n_pool, dtype=torch.int32, device="cuda").index_add_(0, word_cb, bad_w)
                err[m] += int((per_cb > 0).sum())
                iters[m] += int((o["status"] & 0xFFFF).sum())
                if n_done < args.sweep_oracle_n:
                    same[m].append(per_cb > 0)
            if n_done < args.sweep_oracle_n:
                n_take = min(n_pool, args.sweep_oracle_n - n_done)
                tb_take = int(np.searchsorted(w0.tbs["first_cb"] + w0.tbs["n_cb"], n_take, side="left")) + 1
                wn = subset(w0, range(min(w0.n_tb, tb_take)))
                for m in sess:
                    same[m][-1] = same[m][-1][:wn.n_cb].cpu().numpy()
                wn.sym = y[:wn.sym.size].copy()
                wn.cbs["inv_sigma2"] = cbs["inv_sigma2"][:wn.n_cb]
                per = max(1, wn.n_tb // (4 * cores))
                oracle_jobs.append(pool.map_async(_oracle_errors, [
                    (subset(wn, range(i, min(wn.n_tb, i + per))), mi, et) for i in range(0, wn.n_tb, per)]))
            n_done += n_pool
        o_blk = np.concatenate([np.concatenate(job.get()) for job in oracle_jobs]).astype(bool)
        o_err, o_n = int(o_blk.sum()), int(o_blk.size)
        row = {("es_n0_offset_db" if is_mixed else "es_n0_db"): pt, "n_gpu": n_done, "n_oracle": o_n}
        for m in sess:
            g_blk = np.concatenate(same[m]).astype(bool)
            assert g_blk.size == o_n
            row[m] = {"bler": err[m] / n_done, "ci95": wilson(err[m], n_done), "mean_iters": iters[m] / n_done,
                      "same_noise": {"bler": float(g_blk.mean()), "outcome_equal_frac": float(np.mean(g_blk == o_blk))}}
        row["f64_oracle"] = {"bler": o_err / max(o_n, 1), "ci95": wilson(o_err, o_n)}
        lo, hi = row["f64_oracle"]["ci95"]
        row["f32_inside_oracle_ci"] = bool(lo <= row["f32"]["bler"] <= hi)
        rows.append(row)
        print(json.dumps({"point": row}), flush=True)
    pool.close()
    desc = ("mixed workload shapes (BG1/BG2-shaped, Z 32..384, R 0.3..0.9, QPSK..256-QAM, URLLC masks), "
            "each code block at its shape's operating point + offset" if is_mixed else
            "BG1-shaped Z=384 K=8448 R=1/2 16-QAM with URLLC masks")
    res = {"sweep": "precision", "config": args.config, "workload": desc, "pool_code_blocks": n_pool,
           "points": rows, "wall_s": time.perf_counter() - t_start, "oracle_cores": cores}
    print(json.dumps(res), flush=True)


# ----------------------------------------------------------------------------- serving
def _pct(x, q):
    return float(np.percentile(x, q)) if len(x) else None


def serve_measure(pool_n: int, slots: int, loads, forms, thresholds=(0,), releases=(0,), loops=(1,),
                  plain_n: int = 400, cb_crc: bool = False, punct_sample: int = 0, verbose: bool = True,
                  mode: str = "i8") -> dict:
    """Replay the served request stream through the decode service; latency vs the 125 us slot.

    40 UEs, Poisson TB requests per 125 us slot (``loads``: TBs per UE per slot, 1.0 = the configuration's
    rate), TBs of 1-16 code blocks of the mixed shapes drawn from a pool of pre-encoded TBs; per slot one
    URLLC codebook entry on the slot's shared subcarrier grid, expanded on the device; INT8 service.
    Beside it, the FP32 unbatched plain path: one TB at a time through puncture_demap + decode_batch +
    tb_crc_goodput, synchronised, on the first requests of the stream at the last load (masks expanded on
    the host).
    """
    import torch
    from paper_2506_00167_gb300 import Server, Session, abi
    from workload.configs import subset
    from workload.serving import (CODEBOOK_PRB, SLOT_NS, codebook_bitmaps, expand_mask, pool_bytes,
                                  served_workload, slot_stream, tb_pool, tb_records)

    torch.cuda.set_device(0)
    t_gen = time.perf_counter()
    w = tb_pool(pool_n, seed=5, cb_crc=cb_crc)
    book = codebook_bitmaps()
    raw, mask_base = pool_bytes(w)
    host = torch.from_numpy(raw).pin_memory()
    gen_s = time.perf_counter() - t_gen
    first = w.tbs["first_cb"].astype(np.int64)
    kbits = np.array([w.bgs[int(b)].kb for b in w.cbs["bg"][first]], np.int64) * \
        w.cbs["Z"][first].astype(np.int64) * w.tbs["n_cb"].astype(np.int64)
    sess = Session(w.bgs, w.z_set, mode=mode, max_iter=10, early_term=True, sat=SAT[mode])
    curves = {}
    streams = {load: slot_stream(slots, w.tbs["n_sc"], n_ue=40, tb_per_slot=load, seed=6) for load in loads}
    runs = [(f, lp, th, rl) for f in forms for lp in loops
            for th in (thresholds if f == "auto" else [0])
            for rl in (releases if f == "auto" else [0])]
    for form, lps, thr, rel in runs:
        srv = Server(sess, host, None, arena_bytes=8 << 30, max_inflight=16384, idle_timeout_us=200000,
                     loops_per_sm=lps, cb_crc=cb_crc, paired=SERVE_FORMS[form], pair_threshold=thr,
                     pair_release=rel, codebook=(book, CODEBOOK_PRB))
        # warm-up
        st0 = streams[loads[0]]
        warm = tb_records(w, mask_base, abi.SERVE_TB_NP, pool_index=st0["pool"][:64], pattern=st0["pattern"][:64],
                          grid_sc=st0["grid_sc"][:64])
        srv.replay(warm, np.zeros(warm.size, np.int64), timeout_ms=30000)
        pts = []
        for load in loads:
            st = streams[load]
            recs = tb_records(w, mask_base, abi.SERVE_TB_NP, pool_index=st["pool"], pattern=st["pattern"],
                              grid_sc=st["grid_sc"])
            c0 = srv.stats()
            t0 = time.perf_counter()
            done = srv.replay(recs, st["t_ns"], timeout_ms=60000)
            wall = time.perf_counter() - t0
            c1 = srv.stats()
            lat_us = (done["t_complete_ns"] - done["t_submit_ns"]) / 1e3
            bits = int(kbits[st["pool"]].sum())
            span = (int(done["t_complete_ns"].max()) - int(done["t_submit_ns"].min())) / 1e9  # first arrival -> last completion
            pts.append({"form": form, "pair_threshold": thr, "pair_release": rel, "loops_per_sm": lps,
                        "tb_per_ue_per_slot": load, "slots": slots, "requests": int(recs.size),
                        "code_blocks": int(recs["n_cb"].sum()),
                        "offered_gbps": bits / (slots * SLOT_NS / 1e9) / 1e9,
                        "served_gbps": bits / span / 1e9, "span_s": span, "wall_s": wall,
                        "p50_us": _pct(lat_us, 50), "p99_us": _pct(lat_us, 99), "p999_us": _pct(lat_us, 99.9),
                        "max_us": float(lat_us.max()), "within_slot_frac": float(np.mean(lat_us <= 125.0)),
                        "tb_crc_ok_frac": float(np.mean(done["d"])),
                        "mean_max_iters": float(np.mean(done["max_iters"])),
                        "items_single": int(c1["items_single"] - c0["items_single"]),
                        "items_paired": int(c1["items_paired"] - c0["items_paired"]),
                        "loop_launches": int(c1["launches"] - c0["launches"]),
                        "host_longest_pass_us": c1["replay_longest_pass_ns"] / 1e3,
                        "host_passes_over_1ms": int(c1["replay_passes_over_1ms"]),
                        "host_longest_pass_at_ms": c1["replay_longest_pass_at_ns"] / 1e6,
                        "host_involuntary_switches": int(c1["replay_involuntary_switches"]),
                        "host_voluntary_switches": int(c1["replay_voluntary_switches"]),
                        "host_minor_faults": int(c1["replay_minor_faults"]),
                        "host_major_faults": int(c1["replay_major_faults"]),
                        **_stall_stats(done)})
            if verbose:
                print(json.dumps({"serving_point": pts[-1]}), flush=True)
        srv.stop()
        curves[f"{form}{thr or ''}{'-' + str(rel) if rel else ''}_{lps}_loops_per_sm"] = pts
    # FP32 unbatched plain path: one TB at a time, synchronised (plain_n = 0: not run)
    plain = None
    if plain_n > 0:
        st = streams[loads[-1]]
        n_plain = min(plain_n, st["pool"].size)
        sw = served_workload(w, st["pool"][:n_plain], st["pattern"][:n_plain], st["grid_sc"][:n_plain], book)
        sess32 = Session(w.bgs, w.z_set, mode="f32", max_iter=10, early_term=True)
        per = []
        for t in range(n_plain):
            sub = subset(sw, [t])
            b = sess32.batch(sub.cbs, sub.tbs, sub.slot_N)
            sym = torch.from_numpy(sub.sym.astype(np.complex64)).cuda()
            mask = torch.from_numpy(sub.mask.view(np.int32)).cuda()
            per.append((b, sym, mask, b.alloc_outputs(), int(kbits[st["pool"][t]])))
        for b, sym, mask, out, _ in per[:8]:
            sess32.run(b, sym, mask, out)
        torch.cuda.synchronize()
        lat, oks = [], []
        tot_bits = 0
        t0 = time.perf_counter()
        for b, sym, mask, out, kb in per:
            t1 = time.perf_counter()
            sess32.run(b, sym, mask, out)
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - t1) * 1e6)
            tot_bits += kb
        wall = time.perf_counter() - t0
        for b, sym, mask, out, _ in per:
            oks.append(int(out["d"][0].item()))
        plain = {"mode": "f32", "tbs": n_plain, "gbps": tot_bits / wall / 1e9, "p50_us": _pct(lat, 50),
                 "p99_us": _pct(lat, 99), "p999_us": _pct(lat, 99.9), "tb_crc_ok_frac": float(np.mean(oks))}
    res = {"workload": "40 UEs, Poisson TB requests per 125 us slot, TBs of 1-16 code blocks of the mixed "
                       "shapes; per slot one entry of a 128-entry URLLC codebook (7 mini-slot bits, "
                       "q = 1 - 0.92^12; 4-12-PRB runs on a 66-PRB period) on the slot's shared grid, "
                       f"expanded on the device; {dict(i8='INT8', f32='FP32', i16='INT16')[mode]} service",
           "cb_crc": bool(cb_crc), "forms": list(forms), "slots_per_load": slots, "pool_tbs": w.n_tb,
           "pool_gen_s": gen_s, "loads": curves, "fp32_unbatched_plain": plain}
    if punct_sample:
        st = streams[loads[-1]]
        hit = tot = 0
        for t, p_, g in zip(st["pool"][:punct_sample], st["pattern"][:punct_sample], st["grid_sc"][:punct_sample]):
            for words in expand_mask(w, int(t), int(p_), int(g), book):
                hit += int(np.unpackbits(words.view(np.uint8)).sum())
            c = w.cbs[int(w.tbs[t]["first_cb"])]
            tot += int(w.tbs[t]["n_cb"]) * (int(c["E"]) // int(c["Qm"]))
        res["punctured_re_frac"] = {"value": hit / tot, "sample_requests": int(punct_sample)}
    if os.environ.get("LDPCGB_CHECKED") == "1":  # checked library: the first failed device index check, if any
        log = (ctypes.c_uint32 * 8)()
        abi.check(abi.load().ldpc_check_log(log), "ldpc_check_log")
        res["check_log"] = list(log)
    return res


def latency_floor(reps: int = 20) -> dict:
    """One code block alone on the GPU, running all 10 iterations: the per-block decode latency that bounds the
    service's tail.  BG1-shaped Z=384 at R=1/3 (all 46 rows) and R=1/2 (24 rows), QPSK below the waterfall so
    that no early exit happens; through the batch decoder (FP32, INT16, INT8) and as a lone request to the INT8
    service in each form (symbols demapped from pinned host memory, CRC included)."""
    import torch
    from paper_2506_00167_gb300 import Server, Session, abi
    from workload.configs import TBSpec, build, default_bgs, es_n0_sigma2
    from workload.serving import pool_bytes, tb_records

    bgs = default_bgs()
    out = {}
    for R, snr in ((1 / 3, -2.0), (0.5, 2.0)):
        Z, Qm = 384, 2
        E = Qm * int(round(bgs[0].kb * Z / (R * Qm)))
        width = 12 * (-(-(E // Qm) // 168))
        w = build("one", bgs, [TBSpec(0, 0, Z, Qm, E, 1, float(es_n0_sigma2(snr)), 0, width)], [width],
                  [np.zeros((14, width), bool)], seed=5)
        m_eff = bgs[0].m_eff(Z, E)
        sym = torch.from_numpy(w.sym.astype(np.complex64)).cuda()
        mask = torch.from_numpy(w.mask.view(np.int32)).cuda()
        tag = f"R{R:.2f}"
        for mode in ("f32", "i16", "i8"):
            s = Session(w.bgs, w.z_set, mode=mode, max_iter=10, early_term=True, sat=SAT[mode])
            b = s.batch(w.cbs, w.tbs, w.slot_N)
            o = b.alloc_outputs()
            s.puncture_demap(b, sym, mask, o["llr"])
            for _ in range(5):
                s.decode_batch(b, o["llr"], o["bits"], o["status"])
            torch.cuda.synchronize()
            st = torch.cuda.current_stream()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                s.decode_batch(b, o["llr"], o["bits"], o["status"])
                e1.record(st)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e3)
            it = int(o["status"][0].item()) & 0xFFFF
            us = float(np.median(ts))
            out[f"{tag}_{mode}_batch"] = {"us": us, "iters": it, "rows": m_eff, "us_per_iter": us / it,
                                          "us_per_layer": us / it / m_eff}
            for C in (2, 4):  # the same block on a cluster of C CTAs
                for _ in range(3):
                    s.decode_cluster(b, o["llr"], o["bits"], o["status"], C)
                torch.cuda.synchronize()
                tc = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    s.decode_cluster(b, o["llr"], o["bits"], o["status"], C)
                    e1.record(st)
                    torch.cuda.synchronize()
                    tc.append(e0.elapsed_time(e1) * 1e3)
                uc = float(np.median(tc))
                out[f"{tag}_{mode}_cluster{C}"] = {"us": uc, "iters": int(o["status"][0].item()) & 0xFFFF,
                                                   "us_per_layer": uc / it / m_eff}
        raw, mb = pool_bytes(w)
        host = torch.from_numpy(raw).pin_memory()
        s8 = Session(w.bgs, w.z_set, mode="i8", max_iter=10, early_term=True, sat=SAT["i8"])
        for paired in (False, True):
            srv = Server(s8, host, None, arena_bytes=1 << 24, max_inflight=8, paired=paired)
            rec = tb_records(w, mb, abi.SERVE_TB_NP)
            lat = []
            for i in range(reps + 5):
                rec["tag"] = i
                d = srv.replay(rec, np.zeros(1, np.int64), timeout_ms=5000)
                lat.append((int(d["t_complete_ns"][0]) - int(d["t_submit_ns"][0])) / 1e3)
                time.sleep(0.002)
            srv.stop()
            out[f"{tag}_i8_serve_{'paired' if paired else 'single'}"] = {
                "p50_us": float(np.median(lat[5:])), "min_us": float(np.min(lat[5:])), "iters": int(d["max_iters"][0])}
    return out


def run_serving(args):
    res = serve_measure(args.serve_pool, args.serve_slots, args.serve_loads, args.serve_form,
                        args.serve_pair_threshold, args.serve_pair_release, args.serve_loops, args.serve_plain,
                        args.cb_crc, punct_sample=1000, mode=args.serve_mode)
    res["mode"] = args.serve_mode
    res["single_block_latency"] = latency_floor()
    print(json.dumps({"serving": res}), flush=True)


def mixed_measure(steps: int = 10, world: int = 1) -> dict:
    """The uneven batch (S1): the mixed workload's 512 slots (BG1/BG2-shaped, Z 32-384, R 0.3-0.9, QPSK-256-QAM,
    1-8 code blocks per TB, URLLC arrivals) as one CUDA graph per step -- demap, one persistent decoder launch
    over every shape (work queue, autotuned tiles), CRC/goodput -- in INT8 (paired) and FP32."""
    import torch
    from paper_2506_00167_gb300 import Graph, Session

    w = make_workload("mixed")
    mi, et = w.meta["max_iter"], bool(w.meta["early_term"])
    sym = torch.from_numpy(np.ascontiguousarray(w.sym, dtype=np.complex64)).cuda()
    mask = torch.from_numpy(np.ascontiguousarray(w.mask).view(np.int32)).cuda()
    res = {"workload": "mixed: 512 slots x 8 UEs, TBs of 1-8 code blocks, BG1/BG2-shaped, Z 32-384, R 0.3-0.9, "
                       "QPSK-256-QAM, 1-4 URLLC arrivals per slot", "code_blocks": w.n_cb,
           "shapes": len({(int(c["bg"]), int(c["Z"])) for c in w.cbs}), "info_bits_per_step": w.info_bits_total()}
    for mode in ("i8", "f32"):
        s = Session(w.bgs, w.z_set, mode=mode, max_iter=mi, early_term=et, sat=SAT[mode])
        tiles = apply_tiles(s, w, mode, "auto", world)
        b = s.batch(w.cbs, w.tbs, w.slot_N)
        out = b.alloc_outputs()
        g = Graph(s, b, sym, mask, out)
        for _ in range(3):
            g.launch()
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            g.launch()
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        g.close()
        status = out["status"].cpu().numpy()
        res[mode] = {"value": w.info_bits_total() / (ms / 1e3) / 1e9, "unit": "Gbit/s", "ms_per_step": ms,
                     "decoder_launches": len(b.plan()), "mean_iters": float(np.mean(status & 0xFFFF)),
                     "tiles": tiles.get("source")}
        if s.device_errors():
            raise RuntimeError("device error word set in the mixed leg")
    return res


def serve_summary(res: dict) -> dict:
    """The bench line's serving key: the configured load's latency against the 125 us slot."""
    pt = next(iter(res["loads"].values()))[-1]
    keep = ("tb_per_ue_per_slot", "slots", "requests", "offered_gbps", "served_gbps", "p50_us", "p99_us",
            "p999_us", "max_us", "within_slot_frac", "tb_crc_ok_frac", "mean_max_iters", "items_single",
            "items_paired", "host_longest_pass_us", "host_passes_over_1ms", "host_longest_pass_at_ms",
            "host_involuntary_switches", "host_minor_faults", "max_gap_device_us", "max_gap_host_us",
            "max_admit_wait_us")
    return {"workload": res["workload"], "form": pt["form"], **{k: pt[k] for k in keep},
            "slot_us": 125.0, "p99_within_slot": pt["p99_us"] <= 125.0,
            "fp32_unbatched_plain": res["fp32_unbatched_plain"], "pool_tbs": res["pool_tbs"]}


SERVE_FORMS = {"auto": "auto", "paired": True, "single": False}


def _stall_stats(done):
    """Where the time of the slowest requests went: the longest pause between consecutive completions as
    the device wrote them and as the host collected them, and how late the host collected the slowest
    request's completion (relative to the median host-minus-device offset)."""
    td = np.sort(done["t_device_ns"].astype(np.int64))
    th = np.sort(done["t_complete_ns"].astype(np.int64))
    off = done["t_complete_ns"].astype(np.int64) - done["t_device_ns"].astype(np.int64)
    lat = done["t_complete_ns"] - done["t_submit_ns"]
    worst = int(np.argmax(lat))
    admit_wait = (done["t_admit_ns"] - done["t_submit_ns"]) / 1e3
    return {"max_gap_device_us": float(np.diff(td).max() / 1e3) if td.size > 1 else 0.0,
            "max_gap_host_us": float(np.diff(th).max() / 1e3) if th.size > 1 else 0.0,
            "worst_host_lag_us": float((off[worst] - np.median(off)) / 1e3),
            "worst_admit_wait_us": float(admit_wait[worst]), "max_admit_wait_us": float(admit_wait.max())}


# ----------------------------------------------------------------------------- main arm
def run_policy(args):
    """Puncturing allocations for the paper's case-study setting (N = 780 SCs, 10 eMBB users, 300-SC
    URLLC packets): RP and SeF per mini-slot and the per-symbol SC masks for args.policy_tti TTIs, the
    feasibility enforcer over the floor(N/L) = 2 branches of every TTI, the enforcer's latency for one TTI
    (the RT O-DU step, one launch) and its throughput on a large batch; beside them the oracle on a
    bounded sample on the host cores."""
    import torch
    from oracle import policy as OP
    from paper_2506_00167_gb300 import policy as GP
    from workload.policy import branch_samples, schedules

    torch.cuda.set_device(0)
    T = args.policy_tti
    alloc_np, demand_np = schedules(T)
    m_np, n_np, tot_np = branch_samples(alloc_np)
    alloc = torch.from_numpy(alloc_np.astype(np.int32)).cuda()
    demand = torch.from_numpy(demand_np.astype(np.int32)).cuda()
    m, n, tot = (torch.from_numpy(m_np.astype(np.float32)).cuda(), torch.from_numpy(n_np.astype(np.int32)).cuda(),
                 torch.from_numpy(tot_np.astype(np.int32)).cuda())
    words = (780 + 31) // 32

    def dev_ms(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"workload": f"{T} TTIs: N = 780 SCs (65 PRBs), 10 eMBB users, 7 mini-slots, 300-SC URLLC packets "
                       "from 12 users with Bernoulli(0.08) arrivals per mini-slot (at most 2 per mini-slot)"}
    for pol in ["rp", "sef"]:
        pm, _ = GP.puncture_alloc(alloc, demand, pol)
        ms_alloc = dev_ms(lambda: GP.puncture_alloc(alloc, demand, pol), args.steps)
        ms_mask = dev_ms(lambda: GP.sc_mask(alloc, pm, words), args.steps)
        out[pol] = {"alloc_ms": ms_alloc, "mask_ms": ms_mask, "tti_per_s": T / ((ms_alloc + ms_mask) / 1e3),
                    "mask_gbs": T * 14 * words * 4 / (ms_mask / 1e3) / 1e9}
    ms_enf = dev_ms(lambda: GP.enforce(m, n, tot), args.steps)
    out["enforcer"] = {"problems": int(tot_np.size), "batch_ms": ms_enf}
    # one TTI (2 branches) per launch: the RT O-DU step's latency
    m1, n1, t1 = m[:2].contiguous(), n[:2].contiguous(), tot[:2].contiguous()
    lat = []
    for _ in range(200):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        GP.enforce(m1, n1, t1)
        e1.record()
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1) * 1e3)
    host = []
    for _ in range(200):
        t0 = time.perf_counter()
        GP.enforce(m1, n1, t1)
        torch.cuda.synchronize()
        host.append((time.perf_counter() - t0) * 1e6)
    out["enforcer"]["one_tti_events_around_call_us_p50"] = float(np.percentile(lat[20:], 50))
    out["enforcer"]["one_tti_host_roundtrip_us_p50"] = float(np.percentile(host[20:], 50))
    # the kernel alone: 100 one-TTI calls captured in a CUDA graph and replayed back to back
    # (device time per call, inter-kernel gaps included; the binding's host overhead excluded)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            GP.enforce(m1, n1, t1)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(100):
            GP.enforce(m1, n1, t1)
    out["enforcer"]["one_tti_kernel_us"] = dev_ms(lambda: g.replay(), 20) * 1e3 / 100
    # throughput on a large batch
    big = 1 << 20
    reps = -(-big // tot_np.size)
    mb, nb, tb = (m.repeat(reps, 1)[:big].contiguous(), n.repeat(reps, 1)[:big].contiguous(),
                  tot.repeat(reps)[:big].contiguous())
    ms_big = dev_ms(lambda: GP.enforce(mb, nb, tb), 5)
    out["enforcer"]["large_batch"] = {"problems": big, "ms": ms_big, "problems_per_s": big / (ms_big / 1e3)}
    # RT O-DU step (Alg. 2): policy forward pass for both branches + enforcer, one TTI per block
    from workload.policy import actor_noise, actor_weights
    wts = [torch.from_numpy(a).cuda() for a in actor_weights()]
    noise = torch.from_numpy(actor_noise(T)).cuda()
    ms_odu = dev_ms(lambda: GP.rt_odu_codebook(alloc, *wts, noise, 300), args.steps)
    a1, nz1 = alloc[:1].contiguous(), noise[:1].contiguous()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            GP.rt_odu_codebook(a1, *wts, nz1, 300)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2):
        for _ in range(100):
            GP.rt_odu_codebook(a1, *wts, nz1, 300)
    out["rt_odu"] = {"network": "10 + 1 inputs, 128 ReLU hidden, 20 outputs (random weights: timing form)",
                     "batch_ms": ms_odu, "tti_per_s": T / (ms_odu / 1e3),
                     "one_tti_kernel_us": dev_ms(lambda: g2.replay(), 20) * 1e3 / 100,
                     "paper_context": "94.4 us average per TTI for forward pass + enforcer on a V100 (Sec. VII-B)"}
    # oracle, bounded sample
    k = min(2000, tot_np.size)
    t0 = time.perf_counter()
    for p in range(k):
        OP.enforce(m_np[p].astype(np.float32), n_np[p], int(tot_np[p]) // 300, 300)
    cpu_enf = (time.perf_counter() - t0) / k
    t0 = time.perf_counter()
    for t in range(min(1000, T)):
        OP.allocate(alloc_np[t], demand_np[t], "rp")
    cpu_rp = (time.perf_counter() - t0) / min(1000, T)
    out["cpu_oracle"] = {"enforcer_us_per_problem": cpu_enf * 1e6, "rp_us_per_tti": cpu_rp * 1e6, "cores": 1,
                         "sample": f"first {k} enforcer problems, first {min(1000, T)} TTIs (RP), one process"}
    out["paper_context"] = "the paper reports 10-30 us for its enforcer on a V100 (Sec. V-B): context only"
    print(json.dumps({"policy": out}), flush=True)


# ----------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large", choices=["large", "mixed", "tiny"])
    ap.add_argument("--mode", default=None, choices=["f32", "i8", "i16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-int8", action="store_true")
    ap.add_argument("--tiles", default="auto",
                    help="decoder tiles: auto (autotuner cache for this GPU, tuned if absent), default, or a path")
    ap.add_argument("--cpu-tb", type=int, default=4096, help="TBs in the timed CPU-oracle sample")
    ap.add_argument("--cpu-min-s", type=float, default=10.0,
                    help="the CPU-oracle sample is timed over whole passes until this many seconds")
    ap.add_argument("--n", type=int, default=None, help="workload size (code blocks / slots); default full")
    ap.add_argument("--min-warmup-s", type=float, default=1.0,
                    help="keep warming up (untimed) at least this long so clocks settle and are sampled")
    ap.add_argument("--ref-tb", type=int, default=192, help="TBs per step of the reference arm")
    ap.add_argument("--serve", action="store_true", help="replay the served request stream instead")
    ap.add_argument("--serve-mode", choices=["i8", "f32", "i16"], default="i8",
                    help="arithmetic of the decode service (the paired form is INT8 only)")
    ap.add_argument("--serve-form", choices=sorted(SERVE_FORMS), nargs="+", default=["auto"],
                    help="INT8 service: pair code blocks by load (auto), always, or never (single); "
                         "several run one after the other")
    ap.add_argument("--serve-pair-threshold", type=int, nargs="+", default=[0],
                    help="auto form: pair a request when more work items than this would be in flight "
                         "(0: one per loop thread block); several run one after the other")
    ap.add_argument("--serve-pair-release", type=int, nargs="+", default=[0],
                    help="auto form: once pairing, keep pairing until the items in flight fall to this "
                         "(0: the threshold)")
    ap.add_argument("--cb-crc", action="store_true",
                    help="mixed / served TBs of several code blocks carry a CRC per code block (CRC-aided exit)")
    ap.add_argument("--policy", action="store_true", help="time the puncturing allocations (RP, SeF, enforcer)")
    ap.add_argument("--policy-tti", type=int, default=5000)
    ap.add_argument("--serve-slots", type=int, default=100000)
    ap.add_argument("--serve-pool", type=int, default=1024)
    ap.add_argument("--serve-plain", type=int, default=400)
    ap.add_argument("--serve-loads", type=float, nargs="+", default=[0.25, 0.5, 0.75, 1.0])
    ap.add_argument("--serve-loops", type=int, nargs="+", default=[1],
                    help="device loops per SM for the service (1; 2 is withdrawn)")
    ap.add_argument("--no-bench-mixed", dest="bench_mixed", action="store_false",
                    help="leave out the mixed-shape batch key of the benchmark line")
    ap.add_argument("--bench-serve-slots", type=int, default=4000,
                    help="slots of the served stream in the default benchmark line (0: no serving key)")
    ap.add_argument("--sweep", default=None, choices=["precision"],
                    help="run a measurement sweep instead of the benchmark line")
    ap.add_argument("--sweep-n", type=int, default=100000, help="code blocks per SNR point (GPU)")
    ap.add_argument("--sweep-oracle-n", type=int, default=2048, help="code blocks per SNR point (oracle)")
    ap.add_argument("--sweep-pool", type=int, default=4096,
                    help="distinct encoded code blocks (large) or slots of the mixed workload (mixed)")
    ap.add_argument("--sweep-lo", type=float, default=5.5, help="lowest Es/N0 point, dB (10 points, 0.5 dB apart)")
    args = ap.parse_args()
    if args.serve:
        return run_serving(args)
    if args.policy:
        return run_policy(args)
    if args.sweep == "precision":
        return run_precision_sweep(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, world, rank)

    # the oracle pool starts before any CUDA call (spawned workers)
    pool = None
    cores = os.cpu_count() or 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = mp.get_context("spawn").Pool(cores)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2506_00167_gb300 import Session

    w = make_workload(args.config, rank, args.n, args.cb_crc)
    mode = args.mode or w.meta.get("mode", "f32")
    mi, et = w.meta["max_iter"], bool(w.meta["early_term"])
    dev = torch.device("cuda", local)
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    hbm_peak, peak_kind, sm_max_nominal = load_peaks()

    sym_h = torch.from_numpy(np.ascontiguousarray(w.sym, dtype=np.complex64)).pin_memory()
    mask_h = torch.from_numpy(np.ascontiguousarray(w.mask).view(np.int32)).pin_memory()
    sym = sym_h.to(dev)
    mask = mask_h.to(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    tiles_used = {}

    def timed(mode_):
        s = Session(w.bgs, w.z_set, mode=mode_, max_iter=mi, early_term=et, sat=SAT[mode_])
        tiles_used[mode_] = apply_tiles(s, w, mode_, args.tiles, world)
        b = s.batch(w.cbs, w.tbs, w.slot_N)
        out = b.alloc_outputs(local)
        stream = torch.cuda.current_stream(dev)
        for _ in range(args.warmup):
            s.run(b, sym, mask, out)
        torch.cuda.synchronize()
        t_w = time.perf_counter()
        while time.perf_counter() - t_w < args.min_warmup_s:
            for _ in range(4):
                s.run(b, sym, mask, out)
            torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            e_a, e_b, e_c, e_d = ev[k]
            e_a.record(stream)
            s.puncture_demap(b, sym, mask, out["llr"])
            e_b.record(stream)
            s.decode_batch(b, out["llr"], out["bits"], out["status"])
            e_c.record(stream)
            s.tb_crc_goodput(b, out["bits"], out["d"], out["goodput_bits"], out["goodput_sc"], out["reward"])
            e_d.record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = t0.elapsed_time(t1)
        k_ms = {"demap": statistics.mean(e[0].elapsed_time(e[1]) for e in ev),
                "decode": statistics.mean(e[1].elapsed_time(e[2]) for e in ev),
                "crc": statistics.mean(e[2].elapsed_time(e[3]) for e in ev)}
        status = out["status"].cpu().numpy()
        errs = s.device_errors()
        if errs:
            raise RuntimeError(f"device error word {errs:#x}")
        return s, b, out, ms, k_ms, status

    clk = ClockSampler(str(getattr(torch.cuda.get_device_properties(dev), "uuid", local)))
    if not str(clk.gpu_id).startswith("GPU-") and clk.gpu_id.count("-") >= 4:
        clk.gpu_id = "GPU-" + clk.gpu_id
    clk.start()
    s, b, out, ms, k_ms, status = timed(mode)
    clocks = clk.stop()

    # slowest rank, all ranks' decoded bits
    info_bits = w.info_bits_total()
    ms, all_bits = reduce_over_ranks(ms, info_bits * args.steps, world, dev)
    value = all_bits / (ms / 1e3) / 1e9
    ms_step = ms / args.steps

    # ---- the same step as one captured CUDA graph per step
    from paper_2506_00167_gb300 import Graph
    graph = Graph(s, b, sym, mask, out)
    for _ in range(3):
        graph.launch()
    torch.cuda.synchronize()
    barrier()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(torch.cuda.current_stream(dev))
    for _ in range(args.steps):
        graph.launch()
    g1.record(torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    ms_graph = g0.elapsed_time(g1)
    graph.close()

    # ---- end to end through the public API from pinned host buffers: every step copies its inputs in,
    # runs the path and copies its results out; steps alternate between two streams (each with its own
    # batch and device buffers) so one step's copies overlap the other's kernels
    b2 = s.batch(w.cbs, w.tbs, w.slot_N)
    pipes = [(sym, mask, out, b), (torch.empty_like(sym), torch.empty_like(mask), b2.alloc_outputs(local), b2)]
    res_h = [{k: torch.empty_like(o[k], device="cpu").pin_memory() for k in ("d", "goodput_bits", "reward")}
             for _, _, o, _ in pipes]
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    stream = torch.cuda.current_stream(dev)

    def e2e_step(i):
        k = i % 2
        sy, mk, o, bb = pipes[k]
        with torch.cuda.stream(streams[k]):
            sy.copy_(sym_h, non_blocking=True)
            mk.copy_(mask_h, non_blocking=True)
            s.run(bb, sy, mk, o)
            for key in res_h[k]:
                res_h[k][key].copy_(o[key], non_blocking=True)

    for i in range(4):
        e2e_step(i)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st in streams:
        st.wait_event(e0)
    for i in range(args.steps):
        e2e_step(i)
    for st in streams:
        stream.wait_stream(st)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e, e2e_bits = reduce_over_ranks(e0.elapsed_time(e1), info_bits * args.steps, world, dev)
    e2e_val = e2e_bits / (ms_e2e / 1e3) / 1e9
    h2d = sym_h.numel() * 8 + mask_h.numel() * 4
    d2h = sum(t.numel() * t.element_size() for t in res_h[0].values())

    # ---- roofline of the dominant kernel (the decoder)
    eu = edge_updates(w, status)
    mhz = (clocks or {}).get("sm_mhz") or sm_max_nominal
    peak_g = peak_alu_gops(num_sms, mhz)
    achieved_g = ALU_OPS_PER_EDGE * eu / (k_ms["decode"] / 1e3) / 1e9
    hb = hbm_bytes(w, mode)
    roof = {"bound": "alu", "achieved": achieved_g, "peak": peak_g, "unit": "Glaneop/s",
            "frac": achieved_g / peak_g, "traffic": decoder_traffic(mode, w.n_cb, args.config),
            "traffic_source": "profiles/decode_traffic.json (ncu dram bytes, 2048-block capture scaled to the launch)",
            "kernel": "oms_decode_kernel", "launch_ms": k_ms["decode"],
            "edge_updates_per_launch": eu, "alu_ops_per_edge_update": ALU_OPS_PER_EDGE,
            "peak_basis": f"ALU pipe: {num_sms} SMs x {ALU_LANES_PER_SM} lanes x {mhz:.0f} MHz "
                          "(median SM clock sampled from warm-up through the timed region)",
            "hbm_achieved_gbs": hb["decode"] / (k_ms["decode"] / 1e3) / 1e9,
            "hbm_peak_gbs": hbm_peak, "hbm_frac": hb["decode"] / (k_ms["decode"] / 1e3) / 1e9 / hbm_peak,
            "hbm_peak_kind": peak_kind}
    demap_gbs = hb["demap"] / (k_ms["demap"] / 1e3) / 1e9
    kernels = {k: {"ms": v, "share": v / sum(k_ms.values())} for k, v in k_ms.items()}
    kernels["demap"]["hbm_gbs"] = demap_gbs
    kernels["demap"]["hbm_frac"] = demap_gbs / hbm_peak

    # ---- INT8 on the same workload
    int8 = None
    if not args.no_int8 and mode != "i8":
        s8, b8, out8, ms8, k8, st8 = timed("i8")
        int8 = {"value": world * info_bits * args.steps / (ms8 / 1e3) / 1e9, "unit": "Gbit/s",
                "ms_per_step": ms8 / args.steps, "decode_ms": k8["decode"],
                "mean_iters": float(np.mean(st8 & 0xFFFF))}
        del s8, b8, out8

    # ---- the uneven batch (mixed shapes) as one graph per step, and the served stream at the configured load
    mixed_res = mixed_measure(world=world) if (world == 1 and args.config == "large" and args.bench_mixed) else None
    serve = None
    if world == 1 and args.bench_serve_slots > 0:
        serve = serve_summary(serve_measure(256, args.bench_serve_slots, [1.0], ["auto"], plain_n=200,
                                            verbose=False))
        # the same stream through an FP32 service (one code block per thread group; no paired form)
        s32 = serve_summary(serve_measure(256, args.bench_serve_slots, [1.0], ["auto"], plain_n=0, verbose=False,
                                          mode="f32"))
        serve["fp32_service"] = {k: s32[k] for k in ("served_gbps", "p50_us", "p99_us", "p999_us", "within_slot_frac",
                                                     "tb_crc_ok_frac", "mean_max_iters", "host_longest_pass_us")}

    # ---- CPU baseline: the oracle on a bounded sample, all host cores
    cpu = None
    if pool is not None:
        chunks = oracle_sample(w, args.cpu_tb, cores)
        bits = dt = 0.0
        passes = 0
        while passes == 0 or dt < args.cpu_min_s:  # whole passes over the sample until the time is reached
            b_, d_ = time_oracle(pool, chunks, "f64", mi, et)
            bits += b_
            dt += d_
            passes += 1
        pool.close()
        cpu = {"value": bits / dt / 1e9, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
               "sample": f"first {min(args.cpu_tb, w.n_tb)} TBs of the workload, {passes} passes, float64 "
                         f"oracle (demap + decode + CRC), {cores} spawned processes, {dt:.1f} s wall"}

    gpu_launches = args.steps * (2 + len(b.plan()))  # demap + decoder launches + CRC/goodput per step
    line = {"metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"f32": "f32", "i8": "i8", "i16": "i16"}[mode],
            "data": "synthetic (seeded Tx chain: CRC-24, QC-LDPC encode, 16-QAM, AWGN, URLLC puncture masks)",
            "config": {"workload": workload_desc(args),
                       "cb_crc": bool(args.cb_crc),
                       "code_blocks": w.n_cb, "transport_blocks": w.n_tb, "info_bits_per_step": info_bits,
                       "mean_iters": float(np.mean(status & 0xFFFF)),
                       "l2": "inputs larger than L2 (symbols %.0f MB + LLRs %.0f MB per step)"
                             % (w.sym.size * 8 / 1e6, hb["decode"] / 1e6),
                       "parallelism": f"replicas x{world}", "tiles": tiles_used.get(mode)},
            "codewords_per_s": world * w.n_cb * args.steps / (ms / 1e3),
            "graph": {"ms_per_step": ms_graph / args.steps,
                      "value": world * info_bits * args.steps / (ms_graph / 1e3) / 1e9, "unit": "Gbit/s",
                      "decoder_launches": len(b.plan())},
            "kernels": kernels, "roofline": roof, "cpu_baseline": cpu, "int8": int8, "mixed": mixed_res,
            "serve": serve,
            "e2e": {"value": e2e_val, "unit": "Gbit/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "pipeline": "steps alternate over 2 streams: one step's host copies overlap the other's kernels"},
            "gpu_launches": gpu_launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
