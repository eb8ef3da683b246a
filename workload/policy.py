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
