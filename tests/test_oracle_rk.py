"""Pins of the oracle's Runge-Kutta machinery against mathematics (CPU only).

Nothing here re-types the oracle's formulas: the tableau is checked through
Butcher's order conditions generated from rooted trees, the steppers through
their stability functions and quadrature exactness, and the controller through
the tol^(-1/5) work law of an order-5 pair and exact phase-end arrival.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


# ---------------------------------------------------------------------------
# Butcher order conditions from rooted trees
# ---------------------------------------------------------------------------

def _trees(order):
    """All rooted trees with `order` vertices, each a sorted tuple of child trees."""
    if order == 1:
        return [()]
    out = set()

    def partitions(n, max_part):
        if n == 0:
            yield []
            return
        for k in range(min(n, max_part), 0, -1):
            for rest in partitions(n - k, k):
                yield [k] + rest

    for parts in partitions(order - 1, order - 1):
        choices = [_trees(k) for k in parts]

        def build(i, acc):
            if i == len(parts):
                out.add(tuple(sorted(acc)))
                return
            for t in choices[i]:
                build(i + 1, acc + [t])

        build(0, [])
    return sorted(out)


def _size(t):
    return 1 + sum(_size(c) for c in t)


def _gamma(t):
    g = _size(t)
    for c in t:
        g *= _gamma(c)
    return g


def _phi(t, A):
    """Stage vector of elementary weights Phi_i(t)."""
    s = A.shape[0]
    v = np.ones(s)
    for c in t:
        v = v * (A @ _phi(c, A))
    return v


def test_tree_counts():
    assert [len(_trees(k)) for k in range(1, 6)] == [1, 1, 2, 4, 9]


def test_cashkarp_row_sums():
    c, A, b, bs = oracle.cashkarp_tableau()
    np.testing.assert_allclose(A.sum(axis=1), c, rtol=0, atol=2e-16)
    assert np.all(np.triu(A) == 0.0)          # explicit


def test_cashkarp_fifth_order_weights():
    """b satisfies all 17 order conditions through order 5."""
    c, A, b, bs = oracle.cashkarp_tableau()
    for k in range(1, 6):
        for t in _trees(k):
            assert abs(b @ _phi(t, A) - 1.0 / _gamma(t)) < 4e-16, (k, t)


def test_cashkarp_fourth_order_embedded_weights():
    """bs satisfies the 8 conditions through order 4 and misses order 5."""
    c, A, b, bs = oracle.cashkarp_tableau()
    for k in range(1, 5):
        for t in _trees(k):
            assert abs(bs @ _phi(t, A) - 1.0 / _gamma(t)) < 4e-16, (k, t)
    miss = max(abs(bs @ _phi(t, A) - 1.0 / _gamma(t)) for t in _trees(5))
    assert miss > 1e-4


def test_cashkarp_weights_are_the_nearest_doubles_of_rationals():
    """Each weight is a short rational (denominator <= 2^17) rounded once."""
    c, A, b, bs = oracle.cashkarp_tableau()
    for x in list(c) + list(A.ravel()) + list(b) + list(bs):
        f = Fraction(x).limit_denominator(1 << 17)
        assert float(f) == x


# ---------------------------------------------------------------------------
# RK4
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("z", [-0.5, -0.1, 0.05, 0.3, -2.0])
def test_rk4_stability_function(z):
    """One step on y' = lambda y multiplies by R(z) = sum_{k<=4} z^k / k!."""
    y1 = oracle.rk4_step(oracle.LINEAR, [z], 0.0, 1.0, [1.0])[0]
    R = sum(Fraction(z) ** k / math.factorial(k) for k in range(5))
    assert abs(y1 - float(R)) <= 4 * np.spacing(abs(float(R)))


def test_rk4_exact_for_cubic_quadrature():
    """y' = c t^3 reduces RK4 to Simpson's rule, exact for cubics."""
    t0, h, c = 0.3, 0.25, 1.7
    y1 = oracle.rk4_step(oracle.TPOW, [3.0, c], t0, h, [0.0])[0]
    exact = c * ((t0 + h) ** 4 - t0 ** 4) / 4
    assert abs(y1 - exact) <= 4 * np.spacing(exact)


def test_rk4_simpson_error_for_quartic():
    """For y' = t^4 the one-step error equals Simpson's error h^5/120 exactly."""
    t0, h = 0.0, 0.5
    y1 = oracle.rk4_step(oracle.TPOW, [4.0, 1.0], t0, h, [0.0])[0]
    exact = ((t0 + h) ** 5 - t0 ** 5) / 5
    assert abs((y1 - exact) - h ** 5 / 120) < 1e-15


def test_rk4_global_order_four():
    """Global error on y' = -y over [0, 2] drops 16x per halving of h."""
    errs = []
    for nsteps in (20, 40, 80):
        y, st = oracle.rk4_solve(oracle.LINEAR, [[-1.0]], [[1.0]], 0.0, 2.0 / nsteps, nsteps)
        errs.append(abs(y[0, 0] - math.exp(-2.0)))
    for e0, e1 in zip(errs, errs[1:]):
        assert 15.0 < e0 / e1 < 17.0


# ---------------------------------------------------------------------------
# Cash-Karp stepper
# ---------------------------------------------------------------------------

def test_cashkarp_quadrature_exactness():
    """b integrates t^4 exactly; bs integrates t^3 exactly but not t^4."""
    t0, h = 0.2, 0.5
    y5, err = oracle.cashkarp_step(oracle.TPOW, [4.0, 1.0], t0, h, [0.0])
    assert abs(y5[0] - ((t0 + h) ** 5 - t0 ** 5) / 5) < 1e-16
    assert abs(err[0]) > 1e-6                      # the order-4 weights miss t^4
    y5, err = oracle.cashkarp_step(oracle.TPOW, [3.0, 1.0], t0, h, [0.0])
    assert abs(y5[0] - ((t0 + h) ** 4 - t0 ** 4) / 4) < 1e-16
    assert abs(err[0]) < 1e-16


def test_cashkarp_local_orders_on_linear_problem():
    """Local error of y5 is O(h^6), of the embedded y4 O(h^5)."""
    def errs(h):
        y5, err = oracle.cashkarp_step(oracle.LINEAR, [-1.0], 0.0, h, [1.0])
        e5 = y5[0] - math.exp(-h)
        e4 = (y5[0] - err[0]) - math.exp(-h)
        return e5, e4
    a5, a4 = errs(0.05)
    b5, b4 = errs(0.025)
    assert 55 < a5 / b5 < 72            # 2^6 = 64
    assert 28 < a4 / b4 < 37            # 2^5 = 32


# ---------------------------------------------------------------------------
# controller
# ---------------------------------------------------------------------------

def _linear_run(tolv, t1=10.0):
    tol = oracle.make_tol(rtol=tolv, atol=tolv, dt0=1e-3, dt_min=1e-14, dt_max=1.0, t0=0.0, t1=t1)
    return oracle.cashkarp_solve(oracle.LINEAR, [[-1.0]], [[1.0]], tol)


def test_controller_work_scales_as_tol_to_minus_one_fifth():
    """On y' = y (pure relative tolerance) the step is fixed by h^5 ~ tol."""
    steps, errs = [], []
    for tv in (1e-6, 1e-8, 1e-10, 1e-12):
        tol = oracle.make_tol(rtol=tv, atol=0.0, dt0=1e-3, dt_min=1e-14, dt_max=1.0, t0=0.0, t1=20.0)
        r = oracle.cashkarp_solve(oracle.LINEAR, [[1.0]], [[1.0]], tol)
        steps.append(int(r["nacc"][0]))
        errs.append(abs(r["y"][0, 0] / math.exp(20.0) - 1.0))
    for s0, s1 in zip(steps, steps[1:]):
        assert 100 ** 0.2 * 0.9 < s1 / s0 < 100 ** 0.2 * 1.1, steps
    for e, tv in zip(errs, (1e-6, 1e-8, 1e-10, 1e-12)):
        assert tv / 100 < e < 20 * tv, errs


def test_controller_hits_end_and_meets_tolerance():
    r = _linear_run(1e-10)
    assert r["t"][0] == 10.0
    assert r["status"][0] == 0
    # global error of a tolerance-proportional controller stays near tol
    assert abs(r["y"][0, 0] - math.exp(-10.0)) < 1e-9
    assert 1e-14 <= r["dt"][0] <= 1.0


def test_controller_dt_bounds_and_underflow():
    tol = oracle.make_tol(rtol=1e-10, atol=1e-10, dt0=1e-3, dt_min=1e-14, dt_max=0.01, t0=0.0, t1=1.0)
    r = oracle.cashkarp_solve(oracle.LINEAR, [[-1.0]], [[1.0]], tol)
    assert r["nacc"][0] >= 100                    # dt_max = 0.01 caps the step
    # an impossible tolerance drives dt below dt_min and is reported, not hung
    # (y' = t^4: the embedded weights miss t^4, so err never rounds to zero)
    tol = oracle.make_tol(rtol=1e-30, atol=1e-30, dt0=1e-3, dt_min=1e-6, dt_max=0.1, t0=0.0, t1=1.0)
    r = oracle.cashkarp_solve(oracle.TPOW, [[4.0], [1.0]], [[0.0]], tol)
    assert r["status"][0] & oracle.ST_DT_UNDERFLOW


def test_controller_max_steps_status():
    tol = oracle.make_tol(rtol=1e-12, atol=1e-12, dt0=1e-3, dt_min=1e-14, dt_max=1.0, t0=0.0,
                          t1=100.0, max_steps=50)
    r = oracle.cashkarp_solve(oracle.LINEAR, [[-1.0]], [[1.0]], tol)
    assert r["status"][0] & oracle.ST_MAX_STEPS
    assert r["nacc"][0] + r["nrej"][0] == 50


def test_rhs_evaluation_count_reuses_k1_after_rejection():
    r = _linear_run(1e-10)
    n_trials = r["nacc"][0] + r["nrej"][0]
    # 6 evaluations per trial, minus the first stage of every retried trial
    assert r["nrhs"][0] == 6 * n_trials - r["nrej"][0]


def test_single_thread_call_leaves_the_thread_default_alone():
    """nthreads applies to one call only (the timed baselines rely on it)."""
    before = oracle.max_threads()
    y0 = np.array([[1.0, 2.0]])
    oracle.rk4_solve(oracle.LINEAR, np.array([[-1.0, -2.0]]), y0, 0.0, 0.01, 10, nthreads=1)
    assert oracle.max_threads() == before


# ---------------------------------------------------------------------------
# Dormand-Prince 5(4)
# ---------------------------------------------------------------------------

def test_dopri5_row_sums_and_first_same_as_last():
    c, A, b, bs = oracle.dopri5_tableau()
    np.testing.assert_allclose(A.sum(axis=1), c, rtol=0, atol=4e-16)
    assert np.all(np.triu(A) == 0.0)
    # the seventh stage sits at t + h with coupling row b: k7 = f(t + h, y5)
    assert c[6] == 1.0 and np.array_equal(A[6, :6], b[:6]) and b[6] == 0.0


def test_dopri5_fifth_order_weights():
    c, A, b, bs = oracle.dopri5_tableau()
    for k in range(1, 6):
        for t in _trees(k):
            assert abs(b @ _phi(t, A) - 1.0 / _gamma(t)) < 4e-15, (k, t)


def test_dopri5_fourth_order_embedded_weights():
    c, A, b, bs = oracle.dopri5_tableau()
    for k in range(1, 5):
        for t in _trees(k):
            assert abs(bs @ _phi(t, A) - 1.0 / _gamma(t)) < 4e-15, (k, t)
    miss = max(abs(bs @ _phi(t, A) - 1.0 / _gamma(t)) for t in _trees(5))
    assert miss > 1e-5


def test_dopri5_weights_are_the_nearest_doubles_of_rationals():
    c, A, b, bs = oracle.dopri5_tableau()
    for x in list(c) + list(A.ravel()) + list(b) + list(bs):
        f = Fraction(x).limit_denominator(1 << 19)
        assert float(f) == x


def test_dopri5_quadrature_exactness_and_local_orders():
    t0, h = 0.2, 0.5
    y5, err = oracle.dopri5_step(oracle.TPOW, [4.0, 1.0], t0, h, [0.0])
    assert abs(y5[0] - ((t0 + h) ** 5 - t0 ** 5) / 5) < 1e-16
    assert abs(err[0]) > 1e-7
    y5, err = oracle.dopri5_step(oracle.TPOW, [3.0, 1.0], t0, h, [0.0])
    assert abs(y5[0] - ((t0 + h) ** 4 - t0 ** 4) / 4) < 1e-16
    assert abs(err[0]) < 1e-16

    def errs(hh):
        y5, err = oracle.dopri5_step(oracle.LINEAR, [-1.0], 0.0, hh, [1.0])
        return y5[0] - math.exp(-hh), (y5[0] - err[0]) - math.exp(-hh)
    a5, a4 = errs(0.1)
    b5, b4 = errs(0.05)
    assert 55 < a5 / b5 < 72
    assert 28 < a4 / b4 < 37


def test_dopri5_controller_and_first_same_as_last_count():
    """Work law tol^(-1/5), and 1 + 6 evaluations per trial: k1 of an
    accepted step is the previous k7, and a rejected step keeps its k1."""
    steps = []
    for tv in (1e-6, 1e-8, 1e-10):
        tol = oracle.make_tol(rtol=tv, atol=0.0, dt0=1e-3, dt_min=1e-14, dt_max=1.0, t0=0.0, t1=20.0,
                              method=oracle.DOPRI5)
        r = oracle.cashkarp_solve(oracle.LINEAR, [[1.0]], [[1.0]], tol)
        steps.append(int(r["nacc"][0]))
        assert abs(r["y"][0, 0] / math.exp(20.0) - 1.0) < 20 * tv
        assert r["nrhs"][0] == 1 + 6 * (r["nacc"][0] + r["nrej"][0])
    for s0, s1 in zip(steps, steps[1:]):
        assert 100 ** 0.2 * 0.9 < s1 / s0 < 100 ** 0.2 * 1.1, steps


def test_dopri5_phase_mode_restarts_k1_each_phase():
    """Phase mode: tau resets at each phase start, so k1 = f(t0, y) is
    evaluated there instead of reusing k7: 1 + 6 trials per phase."""
    tol = oracle.make_tol(rtol=1e-9, atol=1e-9, dt0=1e-2, dt_min=1e-14, dt_max=0.1, n_phases=3,
                          phase_len=1.0, t0=0.0, method=oracle.DOPRI5)
    r = oracle.cashkarp_solve(oracle.LINEAR, [[-0.5]], [[1.0]], tol)
    assert r["status"][0] == 0
    assert r["nrhs"][0] == 3 + 6 * (r["nacc"][0] + r["nrej"][0])
    assert abs(r["y"][0, 0] - math.exp(-1.5)) < 1e-8
