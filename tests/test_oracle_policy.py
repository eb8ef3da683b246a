"""The puncturing-allocation oracle (RP, SeF, feasibility enforcer) against the paper and the mathematics."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import policy as P

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table6_rp_sef.txt")


def _table6():
    rows = {}
    for ln in open(GOLD):
        ln = ln.strip()
        if ln and not ln.startswith("#"):
            k, *v = ln.split()
            rows[k] = np.array([int(x) for x in v])
    return rows


def test_rp_and_sef_reproduce_table6():
    t = _table6()
    s = t["s"]
    assert s.sum() == 780
    assert np.array_equal(P.rp(s, 300), t["rp_300"])
    assert np.array_equal(P.sef(s, 300), t["sef_300"])
    assert np.array_equal(P.sef(s, 600), t["sef_600"])


def test_rp_600_differs_from_the_printed_column_by_one_sc_between_two_users():
    # The printed RP column for 600 SCs gives user 1 47 SCs (quota 46.15) and user 3 55 (quota 55.38):
    # no rounding of the proportional quotas that keeps the sum (Huntington-Hill, largest remainder,
    # per-packet) gives that; the reading keeps Huntington-Hill, one SC away from the print.
    t = _table6()
    ours = P.rp(t["s"], 600)
    assert ours.sum() == 600 == t["rp_600"].sum()
    d = ours - t["rp_600"]
    assert np.abs(d).sum() == 2 and d[0] == -1 and d[2] == 1


def _hh_cost(a, q):
    # Huntington-Hill minimises sum q_e^2 / a_e (equivalently sum (a_e - q_e)^2 / a_e)
    c = 0.0
    for ae, qe in zip(a, q):
        if qe > 0:
            if ae == 0:
                return math.inf
            c += qe * qe / ae
    return c


def test_hh_round_is_the_minimum_of_its_objective_by_brute_force():
    rng = np.random.default_rng(5)
    for _ in range(300):
        E = int(rng.integers(2, 6))
        q = rng.uniform(0, 9, E) * (rng.random(E) < 0.85)
        T = int(round(q.sum()))
        lo, hi = np.floor(q).astype(int), np.ceil(q).astype(int)
        if not lo.sum() <= T <= hi.sum():
            continue
        a = P.hh_round(q, T)
        assert a.sum() == T and np.all(a >= lo) and np.all(a <= hi)
        best = min(_hh_cost(c, q) for c in itertools.product(*[range(l, h + 1) for l, h in zip(lo, hi)])
                   if sum(c) == T)
        assert math.isclose(_hh_cost(a, q), best, rel_tol=1e-12) or (best == math.inf)


def test_hh_round_special_cases():
    assert np.array_equal(P.hh_round([3.0, 5.0, 2.0], 10), [3, 5, 2])        # integer quotas stay
    assert np.array_equal(P.hh_round([1.5, 1.5], 3), [2, 1])                 # tie: lower index first
    assert np.array_equal(P.hh_round([0.2, 0.2, 0.6], 1), [1, 0, 0])         # a zero seat has top priority
    assert np.array_equal(P.hh_round([2.5, 2.5], 5, cap=[2, 9]), [2, 3])     # caps bind
    with pytest.raises(ValueError):
        P.hh_round([1.2, 1.2], 5)


def test_rp_is_proportional_within_one_sc_and_respects_allocations():
    rng = np.random.default_rng(6)
    for _ in range(200):
        n = rng.integers(12, 200, size=int(rng.integers(2, 12)))
        D = int(rng.integers(1, n.sum() + 1))
        a = P.rp(n, D)
        q = D * n / n.sum()
        assert a.sum() == D and np.all(a <= n) and np.all(np.abs(a - q) < 1)


def test_sef_closed_form():
    n = np.array([30, 10, 20, 10])
    assert np.array_equal(P.sef(n, 15), [0, 10, 0, 5])      # ties: lower index first
    assert np.array_equal(P.sef(n, 45), [5, 10, 20, 10])
    assert np.array_equal(P.sef(n, 70), n)
    with pytest.raises(ValueError):
        P.sef(n, 71)


def test_kl_projection_closed_form_without_caps():
    m = np.array([3.0, 1.0, 0.0, 4.0])
    n = np.array([100.0, 100.0, 100.0, 100.0])
    x = P.kl_project(m, n, 40.0)
    assert np.allclose(x, 40.0 * m / m.sum(), rtol=1e-6, atol=0)


def test_kl_projection_against_a_convex_solver():
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(7)
    for _ in range(40):
        E = int(rng.integers(2, 8))
        n = rng.integers(10, 120, E).astype(float)
        m = rng.uniform(0, 150, E)
        T = float(rng.integers(1, int(n.sum())))
        x = P.kl_project(m, n, T)
        # float32 arithmetic: the sum holds to float32 rounding
        assert math.isclose(float(x.astype(np.float64).sum()), T, rel_tol=1e-5) and np.all(x >= 0) and np.all(x <= n)

        def f(v):
            v = np.maximum(np.asarray(v, dtype=np.float64), 1e-12)
            return float(np.sum(m * np.log(m / v)))
        res = opt.minimize(f, np.full(E, T / E).clip(0, n), method="SLSQP", bounds=list(zip([1e-9] * E, n)),
                           constraints=[{"type": "eq", "fun": lambda v: v.sum() - T}],
                           options={"ftol": 1e-12, "maxiter": 500})
        assert f(x) <= res.fun + 1e-4 * max(1.0, abs(res.fun))


def test_kl_projection_kkt_form_and_zero_users():
    m = np.array([50.0, 0.0, 200.0, 10.0])
    n = np.array([60.0, 30.0, 40.0, 70.0])
    x = P.kl_project(m, n, 90.0)
    # capped user 3 at 40; the others share the rest in proportion to m: c = 50 / 60
    assert np.allclose(x, [50 * 50 / 60, 0.0, 40.0, 10 * 50 / 60], rtol=1e-6, atol=0)
    x = P.kl_project(m, n, 190.0)  # positive users all capped (170); the remaining 20 goes to user 2
    assert np.allclose(x, [60.0, 20.0, 40.0, 70.0], rtol=1e-6, atol=0)


def test_float64_kl_projection_closed_forms_and_convex_solver():
    """The float64 projection (eq. 6 / eq. 7 from its optimality conditions) against closed forms and SLSQP."""
    m = np.array([3.0, 1.0, 0.0, 4.0])
    assert np.allclose(P.kl_project64(m, np.full(4, 100.0), 40.0), 40.0 * m / m.sum(), rtol=1e-14, atol=0)
    m = np.array([50.0, 0.0, 200.0, 10.0])
    n = np.array([60.0, 30.0, 40.0, 70.0])
    assert np.allclose(P.kl_project64(m, n, 90.0), [50 * 50 / 60, 0.0, 40.0, 10 * 50 / 60], rtol=1e-14, atol=0)
    assert np.allclose(P.kl_project64(m, n, 190.0), [60.0, 20.0, 40.0, 70.0], rtol=1e-14, atol=0)
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(17)
    for _ in range(40):
        E = int(rng.integers(2, 8))
        n = rng.integers(10, 120, E).astype(float)
        m = rng.uniform(0, 150, E)
        T = float(rng.integers(1, int(n.sum())))
        x = P.kl_project64(m, n, T)
        assert math.isclose(x.sum(), T, rel_tol=1e-12) and np.all(x >= 0) and np.all(x <= n)

        def f(v):
            v = np.maximum(np.asarray(v, dtype=np.float64), 1e-12)
            return float(np.sum(m * np.log(m / v)))
        res = opt.minimize(f, np.full(E, T / E).clip(0, n), method="SLSQP", bounds=list(zip([1e-9] * E, n)),
                           constraints=[{"type": "eq", "fun": lambda v: v.sum() - T}],
                           options={"ftol": 1e-12, "maxiter": 500})
        assert f(x) <= res.fun + 1e-6 * max(1.0, abs(res.fun))


def test_float64_hh_round_is_the_minimum_of_its_objective_by_brute_force():
    rng = np.random.default_rng(19)
    for _ in range(60):
        E = int(rng.integers(2, 5))
        q = rng.uniform(0.2, 9.0, E)
        total = int(round(q.sum()))
        a = P.hh_round64(q, total)
        best = None
        for cand in itertools.product(*[range(int(math.floor(v)), int(math.ceil(v)) + 1) for v in q]):
            cand = np.array(cand)
            if cand.sum() != total or np.any(cand == 0):
                continue
            obj = float(np.sum(q * q / cand))
            best = obj if best is None else min(best, obj)
        if best is not None and np.all(a > 0):
            assert float(np.sum(q * q / a)) <= best + 1e-9


def test_float32_enforcer_follows_the_float64_reference():
    """The float32 restatement (the arithmetic the CUDA kernel reproduces bit for bit) against the float64
    reference: projections equal to float32 rounding, integer vectors within one unit per user, both
    summing exactly to the demand."""
    rng = np.random.default_rng(23)
    exact = 0
    trials = 0
    for _ in range(400):
        E = int(rng.integers(2, 16))
        n = rng.integers(12, 150, E)
        L = int(rng.integers(20, 120))
        j = int(rng.integers(1, max(2, n.sum() // L) + 1))
        if j * L > n.sum():
            continue
        m = rng.uniform(-0.2, 1.5, E) * n
        m[rng.random(E) < 0.15] = 0.0
        x32 = P.kl_project(m.astype(np.float32), n, j * L).astype(np.float64)
        x64 = P.kl_project64(m.astype(np.float32).astype(np.float64), n, j * L)
        assert np.allclose(x32, x64, rtol=2e-5, atol=2e-5 * j * L)
        a32 = P.enforce(m.astype(np.float32), n, j, L)
        a64 = P.enforce64(m.astype(np.float32).astype(np.float64), n, j, L)
        assert a32.sum() == j * L == a64.sum()
        assert np.all(np.abs(a32 - a64) <= 1) and np.all(a64 <= n) and np.all(a64 >= 0)
        exact += int(np.array_equal(a32, a64))
        trials += 1
    assert exact >= 0.95 * trials, (exact, trials)


def test_enforcer_returns_a_feasible_integer_vector_and_keeps_feasible_ones():
    rng = np.random.default_rng(8)
    for _ in range(200):
        E = int(rng.integers(2, 12))
        n = rng.integers(12, 150, E)
        L = int(rng.integers(20, 120))
        j = int(rng.integers(1, max(2, n.sum() // L) + 1))
        if j * L > n.sum():
            continue
        m = rng.uniform(0, 1.5, E) * n
        a = P.enforce(m, n, j, L)
        assert a.dtype.kind == "i" and a.sum() == j * L and np.all(a >= 0) and np.all(a <= n)
        # an integer vector that is already feasible is its own projection and rounding
        f = P.rp(n, j * L)
        assert np.array_equal(P.enforce(f.astype(float), n, j, L), f)


def test_sc_mask_counts_and_bands():
    n = np.array([60, 108, 72])
    m = np.zeros((7, 3), dtype=int)
    m[1] = [10, 0, 72]
    m[6] = [60, 5, 1]
    msk = P.sc_mask(n, m)
    assert msk.shape == (14, 240)
    assert np.array_equal(msk.sum(axis=1), np.repeat(m.sum(axis=1), 2))
    assert msk[2, :10].all() and not msk[2, 10:60].any() and msk[2, 168:240].all()
    assert msk[12, 60:65].all() and not msk[12, 65:168].any() and msk[13, 168]


def test_softplus_closed_forms():
    v = P.softplus32(np.array([0.0, 30.0, -30.0, 1.0], dtype=np.float32))
    assert np.allclose(v, [math.log(2.0), 30.0, math.exp(-30.0), math.log1p(math.e)], rtol=1e-6, atol=0)


def test_actor_forward_by_hand():
    # x = (0.5, 1); hidden: relu(0 + 0.5 - 1) = 0 and relu(-1 + 0.25 + 2) = 1.25;
    # mu = 0.5 + 1*0 + 2*1.25 = 3; raw sigma 0 -> softplus(0) = ln 2
    w1 = np.array([[1.0, -1.0], [0.5, 2.0]], np.float32)
    b1 = np.array([0.0, -1.0], np.float32)
    w2 = np.array([[1.0, 2.0], [0.0, 0.0]], np.float32)
    b2 = np.array([0.5, 0.0], np.float32)
    a, mu, sg = P.actor_forward([0.5, 1.0], w1, b1, w2, b2, [0.0])
    assert mu[0] == 3.0 and math.isclose(sg[0], math.log(2.0), rel_tol=1e-7)
    assert math.isclose(a[0], (math.tanh(3.0) + 1) / 2, rel_tol=1e-7)      # 0.99752738
    a, _, _ = P.actor_forward([0.5, 1.0], w1, b1, w2, b2, [1.0])          # z = 3 + ln 2
    assert math.isclose(a[0], (math.tanh(3.0 + math.log(2.0)) + 1) / 2, rel_tol=1e-6)


def test_codebook_is_feasible_and_uniform_actions_give_rp():
    s = _table6()["s"]
    E, H = 10, 128
    rng = np.random.default_rng(9)
    w1 = rng.normal(0, 0.3, (H, E + 1)).astype(np.float32)
    b1 = rng.normal(0, 0.1, H).astype(np.float32)
    w2 = rng.normal(0, 0.1, (2 * E, H)).astype(np.float32)
    b2 = rng.normal(0, 0.1, 2 * E).astype(np.float32)
    book, acts = P.rt_odu_codebook(s, w1, b1, w2, b2, rng.normal(size=(2, E)).astype(np.float32), 300)
    assert np.all((acts >= 0) & (acts <= 1))
    assert book[0].sum() == 300 and book[1].sum() == 600 and np.all(book >= 0) and np.all(book <= s)
    # a policy that asks every user for the same fraction of its allocation is RP
    z = np.zeros_like
    b2u = z(b2)
    b2u[:E] = 0.3
    book, _ = P.rt_odu_codebook(s, z(w1), z(b1), z(w2), b2u, np.zeros((2, E), np.float32), 300)
    assert np.array_equal(book[0], P.rp(s, 300)) and np.array_equal(book[1], P.rp(s, 600))
