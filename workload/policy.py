"""Inputs for the puncturing-allocation kernels (input generation only).

The paper's case study (Sec. VII-B, Table IV): N = 780 subcarriers per slot
(65 PRBs of 12), 10 eMBB users, 7 mini-slots, URLLC packets of L = 300 SCs
from 12 URLLC users with Bernoulli(0.08) arrivals per mini-slot.  Per TTI:

* the eMBB schedule s(t): the 65 PRBs split over the 10 users, each at least
  one PRB (a uniform composition), in SCs;
* the URLLC demand per mini-slot: 300 SCs per arrival, at most floor(N / L) = 2
  packets (the enforcer's branch count);
* for the enforcer: a real puncturing vector per branch j, standing in for the
  policy network's sample (no trained weights exist): per user uniform in
  [0, 1.5] x its allocation, rescaled to sum to j L, so some entries exceed
  their allocation and the enforcer has work to do.
"""
from __future__ import annotations

import numpy as np

from .rng import np_stream

N_SC = 780
N_PRB = 65
N_UE = 10
L_URLLC = 300
N_URLLC_UE = 12
P_ARRIVAL = 0.08
N_MINISLOT = 7


def schedules(n_tti: int, seed: int = 7):
    """(alloc int64 [T, 10] SCs, demand int64 [T, 7] URLLC SCs per mini-slot)."""
    rng = np_stream(seed, 21, n_tti)
    cuts = np.sort(np.stack([rng.choice(np.arange(1, N_PRB), N_UE - 1, replace=False) for _ in range(n_tti)]), axis=1)
    edges = np.concatenate([np.zeros((n_tti, 1), np.int64), cuts, np.full((n_tti, 1), N_PRB)], axis=1)
    alloc = 12 * np.diff(edges, axis=1)
    arrivals = (rng.random((n_tti, N_MINISLOT, N_URLLC_UE)) < P_ARRIVAL).sum(axis=2)
    demand = np.minimum(arrivals, N_SC // L_URLLC) * L_URLLC
    return alloc.astype(np.int64), demand.astype(np.int64)


def branch_samples(alloc: np.ndarray, seed: int = 8):
    """Per TTI and branch j = 1 .. floor(N/L): (real vector [T*J, 10], alloc [T*J, 10], total [T*J])."""
    T = alloc.shape[0]
    J = N_SC // L_URLLC
    rng = np_stream(seed, 22, T)
    a = np.repeat(alloc, J, axis=0).astype(np.float64)
    total = np.tile(np.arange(1, J + 1) * L_URLLC, T)
    raw = rng.uniform(0.0, 1.5, size=a.shape) * a
    m = raw * (total / raw.sum(axis=1))[:, None]
    return m, np.repeat(alloc, J, axis=0), total.astype(np.int64)


# ---------------------------------------------------------------------------- link-level case study
QM_CASE = 4      # 16-QAM
R_CASE = 0.5     # BG2-shaped codes at rate 1/2: 5 Z resource elements per code block
CASE_Z = (32, 64, 128, 256, 384)
MAX_CB_CASE = 8


def tb_shape_for_band(width: int):
    """(Z, n_cb) of the TB a user's band carries: BG2-shaped, rate 1/2, 16-QAM, the (Z, n_cb <= 8)
    that fills the most of the band's 14 x width resource elements (ties: fewer, larger code blocks)."""
    avail = 14 * width
    best = None
    for Z in CASE_Z:
        per_cb = 5 * Z
        n = min(MAX_CB_CASE, avail // per_cb)
        if n >= 1 and (best is None or n * per_cb > best[0] or (n * per_cb == best[0] and Z > best[1])):
            best = (n * per_cb, Z, n)
    if best is None:
        raise ValueError("band too narrow for the smallest code block")
    return best[1], best[2]


def case_study(alloc: np.ndarray, masks: list, seed: int = 9, spread_db=(0.0, 3.0)):
    """Link-level TTIs of the paper's case-study setting under given puncture masks.

    alloc: [T, 10] SCs per user (``schedules``); masks[t]: (14, 780) bool punctured REs of TTI t (from a
    puncturing policy).  Each user's band (its SCs after those of the users before it) carries one TB of
    BG2-shaped rate-1/2 16-QAM code blocks (``tb_shape_for_band``) at Es/N0 ~ U[op + lo, op + hi] with
    op the operating point of that rate and modulation; slot width N = 780 SCs.
    """
    from .configs import (N_SYM, TBSpec, build, default_bgs, es_n0_sigma2, operating_point_db)
    bgs = default_bgs()
    rng = np_stream(seed, 23, alloc.shape[0])
    specs, widths, snrs = [], [], []
    E = int(QM_CASE * 5 * 1)  # per Z unit; E = QM * 5Z
    for t in range(alloc.shape[0]):
        sc0 = 0
        for e in range(alloc.shape[1]):
            w = int(alloc[t, e])
            Z, n_cb = tb_shape_for_band(w)
            snr = operating_point_db(R_CASE, QM_CASE) + float(rng.uniform(*spread_db))
            specs.append(TBSpec(t, 1, Z, QM_CASE, E * Z, n_cb, float(es_n0_sigma2(snr)), sc0, w))
            snrs.append(snr)
            sc0 += w
        widths.append(sc0)
    if any(m.shape != (N_SYM, N_SC) for m in masks):
        raise ValueError("masks must be (14, 780)")
    w = build("case_study", bgs, specs, widths, list(masks), seed, snr_db=snrs)
    w.meta.update(dict(name="case_study", max_iter=10, early_term=1, mode="f32", offset=0.5))
    return w


def actor_weights(E: int = N_UE, H: int = 128, seed: int = 10):
    """Random weights of the policy network's shape (no trained weights exist): Glorot-uniform w1 [H, E+1]
    and w2 [2E, H], zero biases except a small negative bias on the raw deviations; float32."""
    rng = np_stream(seed, 24)
    lim1 = np.sqrt(6.0 / (E + 1 + H))
    lim2 = np.sqrt(6.0 / (H + 2 * E))
    w1 = rng.uniform(-lim1, lim1, (H, E + 1)).astype(np.float32)
    w2 = rng.uniform(-lim2, lim2, (2 * E, H)).astype(np.float32)
    b1 = np.zeros(H, np.float32)
    b2 = np.zeros(2 * E, np.float32)
    b2[E:] = -1.0
    return w1, b1, w2, b2


def actor_noise(n_tti: int, J: int = N_SC // L_URLLC, E: int = N_UE, seed: int = 11):
    """Standard-normal draws of the reparameterised samples, [T, J, E] float32."""
    return np_stream(seed, 25, n_tti).standard_normal((n_tti, J, E)).astype(np.float32)
