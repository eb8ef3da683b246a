"""URLLC puncturing allocations: the two benchmark policies and the feasibility enforcer.

TEST INFRASTRUCTURE ONLY (see the package header).

Per mini-slot, a URLLC demand of D subcarriers is taken from the eMBB users'
allocations n_e (the eMBB schedule s(t), Sec. III-A):

* RP, "Resource Proportion" (Sec. VII-A): users lose SCs in proportion to
  n_e.  The quotas q_e = D n_e / sum(n) are made integers summing to D by
  Huntington-Hill rounding (below).
* SeF, "Smallest eMBB First" (Sec. VII-A): users in ascending order of n_e
  (ties: lower index first) lose all their SCs until D is met; the last one
  loses the remainder.
* Feasibility enforcer (Sec. V-B): a real puncturing vector m that may
  exceed the allocations is replaced by the integer vector nearest to it:
  first the projection m^ onto {0 <= m^_e <= n_e, sum m^_e = jL} minimising
  the KL divergence sum_e m_e log(m_e / m^_e) (eq. 6, eq. 7), solved by
  water-filling, then Huntington-Hill rounding of m^ to integers summing to
  jL.

Readings where the paper is silent (each fixed here and in the CUDA path):

* Huntington-Hill rounding keeps every value between its floor and its
  ceiling (the paper: each value is rounded up or down): start from the
  floors and hand the remaining units out one at a time to the largest
  priority q_e / sqrt(a_e (a_e + 1)) (a_e the current value; a_e = 0 gives
  infinite priority), among values still below their ceiling and their cap
  n_e; equal priorities go to the lower index.
* Precision: the paper does not fix one; quotas, priorities and the KL
  projection are float32 (the policy network's output type), every operation
  rounded once and taken in a fixed order.  ``kl_project64``, ``hh_round64``
  and ``enforce64`` state the same enforcer plainly in float64 (the
  projection from the optimality conditions of eq. 7, plain sums); the float32
  form is tested against them (equal to float32 rounding, integer vectors
  within one unit per user, exact sums), and against closed forms, the KKT
  form and a convex solver.
* KL projection: users with m_e > 0 take m^_e = min(n_e, c m_e) with one
  scale c >= 0 (the KKT conditions of eq. 7); users with m_e = 0 take 0 unless
  the others' allocations cannot hold jL, in which case the remainder is
  spread over them in proportion to n_e (their terms of eq. 6 are zero for any
  value, so any split is optimal; this one is the water-filling continuation).
* Subcarriers: user e's band is the n_e subcarriers after those of users
  1 .. e-1 (SC 0 first); the punctured SCs of a mini-slot are the lowest-index
  m_e SCs of the band, in both OFDM symbols of the mini-slot.
"""
from __future__ import annotations

import numpy as np

N_MINISLOT = 7
SYM_PER_MINISLOT = 2


F32 = np.float32


def hh_round(quota, total: int, cap=None) -> np.ndarray:
    """Integers a with sum(a) == total, floor(q) <= a <= ceil(q), a <= cap (Huntington-Hill order)."""
    q = np.asarray(quota, dtype=np.float32)
    n = q.size
    cap = np.full(n, np.iinfo(np.int64).max, dtype=np.int64) if cap is None else np.asarray(cap, dtype=np.int64)
    a = np.minimum(np.floor(q).astype(np.int64), cap)
    hi = np.minimum(np.ceil(q).astype(np.int64), cap)
    left = int(total) - int(a.sum())
    if left < 0 or left > int((hi - a).sum()):
        raise ValueError("no rounding of these quotas sums to the total")
    for _ in range(left):
        best, best_p = -1, F32(-1.0)
        for e in range(n):
            if a[e] >= hi[e]:
                continue
            p = F32(np.inf) if a[e] == 0 else q[e] / np.sqrt(F32(a[e]) * F32(a[e] + 1))
            if p > best_p:  # strict: the lower index keeps a tie
                best, best_p = e, p
        a[best] += 1
    return a


def rp(n, demand: int) -> np.ndarray:
    """Resource Proportion: SCs taken from each user for a demand of `demand` SCs."""
    n = np.asarray(n, dtype=np.int64)
    q = F32(demand) * n.astype(np.float32) / F32(n.sum())
    return hh_round(q, demand, n)


def sef(n, demand: int) -> np.ndarray:
    """Smallest eMBB First: whole allocations, smallest first (lower index on ties)."""
    n = np.asarray(n, dtype=np.int64)
    out = np.zeros_like(n)
    left = int(demand)
    for e in sorted(range(n.size), key=lambda i: (int(n[i]), i)):
        take = min(left, int(n[e]))
        out[e] = take
        left -= take
    if left:
        raise ValueError("demand exceeds the allocations")
    return out


def kl_project(m, n, total) -> np.ndarray:
    """argmin sum_e m_e log(m_e / x_e)  s.t.  0 <= x <= n, sum x = total  (eq. 6, eq. 7), in float32.

    Sums of allocations are integers (exact in any order); sums of m run in
    index order, one float32 operation at a time, so that another
    implementation following the same order reproduces the result bit for
    bit.
    """
    m = np.asarray(m, dtype=np.float32)
    n = np.asarray(n, dtype=np.float32)
    total = F32(total)
    E = m.size
    pos = [e for e in range(E) if m[e] > 0]
    zero = [e for e in range(E) if not m[e] > 0]
    if total > F32(n.astype(np.int64).sum()):
        raise ValueError("total exceeds the allocations")
    x = np.zeros(E, dtype=np.float32)
    cap_pos = F32(sum(int(n[e]) for e in pos))
    if cap_pos <= total:
        # every user with m_e > 0 is capped; the rest goes to the others by capacity
        for e in pos:
            x[e] = n[e]
        rest = total - cap_pos
        cap0 = F32(sum(int(n[e]) for e in zero))
        if rest > 0 and cap0 > 0:
            for e in zero:
                x[e] = rest * n[e] / cap0
        return x
    # water-filling on the scale c: users reach their cap in order of n_e / m_e.
    # With the first k users of that order capped, c_k = (total - their n) /
    # (sum of the other users' m, added in index order); c is the first c_k
    # that leaves the k-th user of the order below its cap.
    order = sorted(pos, key=lambda e: (n[e] / m[e], e))
    rank = {e: k for k, e in enumerate(order)}
    c = F32(0.0)
    for k, e in enumerate(order):
        capped = F32(sum(int(n[f]) for f in pos if rank[f] < k))
        free_m = F32(0.0)
        for f in pos:
            if rank[f] >= k:
                free_m = free_m + m[f]
        c = (total - capped) / free_m
        if c * m[e] <= n[e]:
            break
    for e in pos:
        x[e] = min(n[e], c * m[e])
    return x


def enforce(m, n, j: int, L: int) -> np.ndarray:
    """Feasible integer puncturing vector for branch j (demand j*L SCs)."""
    x = kl_project(m, n, j * L)
    return hh_round(x, j * L, np.asarray(n, dtype=np.int64))


# ---------------------------------------------------------------------------- float64 reference of the enforcer
def kl_project64(m, n, total) -> np.ndarray:
    """The KL projection of eq. 6 / eq. 7 in float64, written from its optimality conditions.

    Minimise sum_e m_e log(m_e / x_e) over 0 <= x_e <= n_e, sum_e x_e = total.
    Stationarity of the Lagrangian gives m_e / x_e = lambda for every user whose
    x_e is strictly inside its box, so x_e = min(n_e, c m_e) with one c = 1 /
    lambda for the users with m_e > 0; c is the value at which these sum to
    the total (the sum is continuous and increasing in c, so it is found
    exactly by walking the breakpoints c = n_e / m_e in increasing order).
    Users with m_e <= 0 contribute nothing to the objective and get 0 unless
    the others' boxes cannot hold the total; then the rest is split over them
    in proportion to n_e.
    """
    m = np.asarray(m, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    total = float(total)
    if total > n.sum():
        raise ValueError("total exceeds the allocations")
    pos = m > 0
    x = np.zeros(m.size)
    if n[pos].sum() <= total:
        x[pos] = n[pos]
        rest = total - n[pos].sum()
        if rest > 0 and n[~pos].sum() > 0:
            x[~pos] = rest * n[~pos] / n[~pos].sum()
        return x
    idx = np.flatnonzero(pos)
    brk = n[idx] / m[idx]                     # c beyond which user e is capped
    order = idx[np.argsort(brk, kind="stable")]
    for k in range(order.size):
        capped, free = order[:k], order[k:]
        c = (total - n[capped].sum()) / m[free].sum()
        if c * m[order[k]] <= n[order[k]]:  # the k-th user stays inside its box: consistent
            break
    x[idx] = np.minimum(n[idx], c * m[idx])
    return x


def hh_round64(quota, total: int, cap=None) -> np.ndarray:
    """Huntington-Hill rounding in float64: floors first, then one unit at a time to the largest
    q / sqrt(a (a + 1)) among values below their ceiling and cap (a = 0: infinite; lower index on ties)."""
    q = np.asarray(quota, dtype=np.float64)
    cap = np.full(q.size, np.iinfo(np.int64).max, dtype=np.int64) if cap is None else np.asarray(cap, np.int64)
    a = np.minimum(np.floor(q).astype(np.int64), cap)
    hi = np.minimum(np.ceil(q).astype(np.int64), cap)
    left = int(total) - int(a.sum())
    if left < 0 or left > int((hi - a).sum()):
        raise ValueError("no rounding of these quotas sums to the total")
    for _ in range(left):
        pri = np.where(a == 0, np.inf, q / np.sqrt(np.maximum(a * (a + 1.0), 1.0)))
        pri[a >= hi] = -np.inf
        a[int(np.argmax(pri))] += 1            # argmax: first (lowest) index among equal priorities
    return a


def enforce64(m, n, j: int, L: int) -> np.ndarray:
    """The feasibility enforcer (Sec. V-B) in float64: KL projection, then Huntington-Hill rounding."""
    return hh_round64(kl_project64(m, n, j * L), j * L, np.asarray(n, dtype=np.int64))


def sc_mask(n, m_per_minislot) -> np.ndarray:
    """(14, sum(n)) bool: punctured subcarriers per OFDM symbol (lowest-index SCs of each band)."""
    n = np.asarray(n, dtype=np.int64)
    m = np.asarray(m_per_minislot, dtype=np.int64).reshape(N_MINISLOT, n.size)
    start = np.concatenate([[0], np.cumsum(n)[:-1]])
    out = np.zeros((N_MINISLOT * SYM_PER_MINISLOT, int(n.sum())), dtype=bool)
    for ms in range(N_MINISLOT):
        for e in range(n.size):
            k = int(m[ms, e])
            if k:
                out[ms * SYM_PER_MINISLOT:(ms + 1) * SYM_PER_MINISLOT, start[e]:start[e] + k] = True
    return out


def allocate(n, demand_per_minislot, policy: str) -> np.ndarray:
    """(7, E) SCs punctured per mini-slot and user under `policy` ('rp' or 'sef')."""
    fn = {"rp": rp, "sef": sef}[policy]
    return np.stack([fn(n, int(d)) if d else np.zeros(len(n), dtype=np.int64) for d in demand_per_minislot])


# ---------------------------------------------------------------------------- RT O-DU actor (timing form)
def softplus32(x):
    """log(1 + e^x) in float32 (numerically safe form)."""
    x = np.asarray(x, dtype=np.float32)
    return (np.maximum(x, F32(0)) + np.log1p(np.exp(-np.abs(x)))).astype(np.float32)


def actor_forward(x, w1, b1, w2, b2, noise):
    """Policy network f_a on one branch input (Sec. VI-B, Sec. VII-B setting): one dense hidden layer,
    ReLU; outputs [mu_1..mu_E, s_1..s_E]; sigma = softplus(s); z = mu + sigma * noise (the
    reparameterisation); action = (tanh(z) + 1) / 2 in [0, 1].  float32; every sum starts at the bias
    and adds the products in index order, each product and sum rounded once.
    Returns (action[E], mu[E], sigma[E])."""
    x = np.asarray(x, dtype=np.float32)
    H = w1.shape[0]
    h = np.zeros(H, dtype=np.float32)
    for k in range(H):
        acc = F32(b1[k])
        for i in range(x.size):
            acc = acc + F32(w1[k, i]) * x[i]
        h[k] = max(acc, F32(0))
    E = w2.shape[0] // 2
    o = np.zeros(2 * E, dtype=np.float32)
    for r in range(2 * E):
        acc = F32(b2[r])
        for k in range(H):
            acc = acc + F32(w2[r, k]) * h[k]
        o[r] = acc
    mu, s = o[:E], o[E:]
    sigma = softplus32(s)
    z = (mu + sigma * np.asarray(noise, dtype=np.float32)).astype(np.float32)
    action = ((np.tanh(z) + F32(1)) / F32(2)).astype(np.float32)
    return action, mu, sigma


def rt_odu_codebook(alloc, w1, b1, w2, b2, noise, L: int):
    """Codebook B*(t) of one TTI (Alg. 2): for branches j = 1 .. J the actor's action on input
    [s(t) / N, j / J], read as the fraction of each user's allocation to puncture, then the
    feasibility enforcer with total j L.  Returns (codebook [J, E] int64, actions [J, E] float32)."""
    alloc = np.asarray(alloc, dtype=np.int64)
    N = int(alloc.sum())
    J = noise.shape[0]
    book = np.zeros((J, alloc.size), dtype=np.int64)
    acts = np.zeros((J, alloc.size), dtype=np.float32)
    for j in range(1, J + 1):
        x = np.concatenate([alloc.astype(np.float32) / F32(N), [F32(j) / F32(J)]]).astype(np.float32)
        a, _, _ = actor_forward(x, w1, b1, w2, b2, noise[j - 1])
        acts[j - 1] = a
        m = (a * alloc.astype(np.float32)).astype(np.float32)
        book[j - 1] = enforce(m, alloc, j, L)
    return book, acts
