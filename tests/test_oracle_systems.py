"""Pins of the oracle's model equations and solvers (CPU only).

Each test checks the oracle against something other than itself: closed-form
solutions, invariant sets, equilibria, an independently derived dimensional
form of the Keller-Miksis equation, its linearisation integrated by SciPy, the
bouncing-ball closed form for the event machinery, and numbers printed in the
paper (tests/golden/).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

WATER_CFG = dict(rho=997.0, c=1497.0, mu=8.9e-4, sigma=0.0725, pv=3166.8, pinf=1.0e5, gamma=1.4)


def _liq(d):
    return oracle.liquid(d["rho"], d["c"], d["mu"], d["sigma"], d["pv"], d["pinf"], d["gamma"])


# ---------------------------------------------------------------------------
# x' = x^2 - p (Sec. 3)
# ---------------------------------------------------------------------------

def _x2p_exact(p, x0, t):
    s = math.sqrt(p)
    if abs(x0) < s:          # x = -s tanh(s (t + C))
        return -s * math.tanh(s * t + math.atanh(-x0 / s))
    # |x0| > s with x0 < 0: x = -s coth(s (t + C))
    u = s * t + math.atanh(s / -x0)
    return -s / math.tanh(u)


@pytest.mark.parametrize("p", [0.1, 0.2, 0.37, 1.0])
def test_x2p_matches_closed_form(p):
    y, st = oracle.rk4_solve(oracle.X2P, [[p]], [[-0.5]], 0.0, 0.01, 1000)
    exact = _x2p_exact(p, -0.5, 10.0)
    assert abs(y[0, 0] - exact) < 1e-9 * abs(exact)
    y2, _ = oracle.rk4_solve(oracle.X2P, [[p]], [[-0.5]], 0.0, 0.02, 500)
    # fourth order: doubling h multiplies the error by ~16
    e1, e2 = abs(y[0, 0] - exact), abs(y2[0, 0] - exact)
    if e1 > 1e-13:           # above rounding level
        assert 10.0 < e2 / e1 < 22.0


# ---------------------------------------------------------------------------
# Lorenz (Sec. 4.1)
# ---------------------------------------------------------------------------

LOR = dict(sigma=10.0, b=8.0 / 3.0)


def _lor_params(rho):
    rho = np.atleast_1d(np.asarray(rho, dtype=float))
    return np.stack([rho, np.full_like(rho, LOR["sigma"]), np.full_like(rho, LOR["b"])])


def test_lorenz_invariant_axis_decays_exponentially():
    """x = y = 0 is invariant and there z' = -b z: RK4 multiplies z by the
    Taylor polynomial R(-b h) each step, and R^N tends to exp(-b t) at order 4."""
    y, _ = oracle.rk4_solve(oracle.LORENZ, _lor_params(15.0), [[0.0], [0.0], [10.0]], 0.0, 0.01, 1000)
    exact = 10.0 * math.exp(-LOR["b"] * 10.0)
    z = -LOR["b"] * 0.01
    rk = 10.0 * (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24) ** 1000
    assert y[0, 0] == 0.0 and y[1, 0] == 0.0
    assert abs(y[2, 0] / rk - 1.0) < 1e-12
    assert abs(y[2, 0] / exact - 1.0) < 5e-7
    y2, _ = oracle.rk4_solve(oracle.LORENZ, _lor_params(15.0), [[0.0], [0.0], [10.0]], 0.0, 0.02, 500)
    assert 12.0 < abs(y2[2, 0] / exact - 1.0) / abs(y[2, 0] / exact - 1.0) < 20.0


@pytest.mark.parametrize("rho", [2.0, 7.5, 13.0, 19.0])
def test_lorenz_rhs_vanishes_at_nontrivial_equilibria(rho):
    s = math.sqrt(LOR["b"] * (rho - 1.0))
    for sign in (1.0, -1.0):
        yy = np.array([[sign * s], [sign * s], [rho - 1.0]])
        dy = oracle.rhs(oracle.LORENZ, _lor_params(rho), 0.0, yy)
        assert np.abs(dy).max() < 1e-13 * max(1.0, rho)


def test_lorenz_long_runs_converge_to_attractors():
    """rho < 1: origin; 1 < rho < 13.9 (no transient chaos): C+ or C-."""
    rho = np.array([0.3, 0.8, 2.0, 5.0, 9.0, 12.0])
    n = rho.size
    y, st = oracle.rk4_solve(oracle.LORENZ, _lor_params(rho), np.full((3, n), 10.0), 0.0, 0.01, 50000)
    assert np.all(st == 0)
    for i, r in enumerate(rho):
        if r < 1.0:
            assert np.abs(y[:, i]).max() < 1e-8
        else:
            s = math.sqrt(LOR["b"] * (r - 1.0))
            target = np.array([math.copysign(s, y[0, i]), math.copysign(s, y[0, i]), r - 1.0])
            assert np.abs(y[:, i] - target).max() < 1e-8


# ---------------------------------------------------------------------------
# Keller-Miksis (Sec. 4.2)
# ---------------------------------------------------------------------------

def test_km_equilibrium_without_driving():
    """P_A = 0: N_KM(1, 0) = C0 - C2 - C3 = 0, so y = (1, 0) is a fixed point.
    The explicit solver runs at the largest step its error test allows, so the
    state wanders off the fixed point only at the tolerance level."""
    liq = _liq(WATER_CFG)
    f = np.array([2e4, 1e5, 1e6])
    C = oracle.km_coefficients(0.0, f, 0.0, 0.0, 0.0, 10e-6, liq)
    assert np.all(C[5:9] == 0.0)
    dy = oracle.rhs(oracle.KM, C, 0.3, np.stack([np.ones(3), np.zeros(3)]))
    assert np.all(np.abs(dy[1]) <= 1e-14 * C[0])
    tol = oracle.make_tol(rtol=1e-10, atol=1e-10, dt0=1e-2, dt_min=1e-14, dt_max=1e-1,
                          n_phases=64, phase_len=1.0, t0=0.0)
    r = oracle.cashkarp_solve(oracle.KM, C, np.stack([np.ones(3), np.zeros(3)]), tol)
    assert np.all(r["status"] == 0)
    assert np.abs(r["acc"] - 1.0).max() < 1e-9
    assert np.abs(r["y"][0] - 1.0).max() < 1e-9


# ---------------------------------------------------------------------------
# Phase mode: the per-phase maximum / minimum rows (Sec. 4.2, Sec. 4.2.1)
# ---------------------------------------------------------------------------
# The paper records, for every forcing period, the largest y1 seen at the
# solver's own step points (no dense output), with tau restarting at 0 each
# period.  The reading implemented: rows 2k and 2k+1 hold the maximum and the
# minimum of y1 over phase k, taken over the accepted step points and the
# phase-start state.  Three problems with closed-form answers pin it.

def _phase_tol(n_phases, dt0=1e-2, dt_max=0.1, tol=1e-10):
    return oracle.make_tol(rtol=tol, atol=tol, dt0=dt0, dt_min=1e-14, dt_max=dt_max,
                           n_phases=n_phases, phase_len=1.0, t0=0.0)


@pytest.mark.parametrize("c", [1.0, -1.0])
def test_phase_rows_of_a_constant_slope(c):
    """y' = c over 5 phases from y0: phase k runs from y0 + c k to
    y0 + c (k + 1).  Row 2k (max) and row 2k+1 (min) are those two values in
    the order the sign of c gives.  This fails if the rows are swapped or
    shifted by one phase, and if the phase-start state is left out (the first
    step point of a phase lies up to dt_max = 0.1 past it)."""
    y0, P = 0.5, 5
    r = oracle.cashkarp_solve(oracle.TPOW, [[0.0], [c]], [[y0]], _phase_tol(P))
    assert r["status"][0] == 0
    acc = r["acc"][:, 0]
    assert acc.size == 2 * P
    for k in range(P):
        start, end = y0 + c * k, y0 + c * (k + 1)
        assert abs(acc[2 * k] - max(start, end)) < 1e-12, (k, acc[2 * k])
        assert abs(acc[2 * k + 1] - min(start, end)) < 1e-12, (k, acc[2 * k + 1])
    assert abs(r["y"][0, 0] - (y0 + c * P)) < 1e-12


def test_phase_rows_restart_tau_every_phase():
    """y' = tau with tau reset to 0 at each phase start adds exactly 1/2 per
    phase, so phase k spans [y0 + k/2, y0 + (k + 1)/2].  Without the reset,
    phase k would add (2k + 1)/2 and the rows of phases 1.. would be off."""
    y0, P = 0.25, 4
    r = oracle.cashkarp_solve(oracle.TPOW, [[1.0], [1.0]], [[y0]], _phase_tol(P))
    assert r["status"][0] == 0
    acc = r["acc"][:, 0]
    for k in range(P):
        assert abs(acc[2 * k] - (y0 + (k + 1) / 2.0)) < 1e-12, (k, acc[2 * k])
        assert abs(acc[2 * k + 1] - (y0 + k / 2.0)) < 1e-12, (k, acc[2 * k + 1])
    assert abs(r["y"][0, 0] - (y0 + P / 2.0)) < 1e-12


def test_phase_rows_of_a_periodic_forcing():
    """y' = cos(2 pi tau): y = y0 + sin(2 pi tau) / (2 pi) peaks at tau = 1/4
    and bottoms out at 3/4, inside each phase.  With dt0 = dt_max = 1/64 every
    step is 1/64 (the local error is far below the tolerance, so the
    controller keeps the largest step), the step points hit 1/4 and 3/4
    exactly, and each phase's rows are y0 + 1/(2 pi) and y0 - 1/(2 pi) to
    the integration error.  Recording only phase ends would give y0 in both
    rows."""
    y0, P = 0.125, 3
    r = oracle.cashkarp_solve(oracle.FCOS, [[1.0]], [[y0]], _phase_tol(P, dt0=1 / 64, dt_max=1 / 64, tol=1e-8))
    assert r["status"][0] == 0
    assert r["nacc"][0] == 64 * P and r["nrej"][0] == 0
    acc = r["acc"][:, 0]
    amp = 1.0 / (2.0 * math.pi)
    for k in range(P):
        assert abs(acc[2 * k] - (y0 + amp)) < 1e-9, (k, acc[2 * k])
        assert abs(acc[2 * k + 1] - (y0 - amp)) < 1e-9, (k, acc[2 * k + 1])
    assert abs(r["y"][0, 0] - y0) < 1e-9


def test_km_tangent_jacobian_matches_central_differences():
    """The hand-derived Jacobian of the tangent system against central
    differences of the plain Keller-Miksis right-hand side (random driven
    states, both frequencies)."""
    rng = np.random.default_rng(17)
    n = 200
    liq = _liq(WATER_CFG)
    C = oracle.km_coefficients(rng.uniform(0, 2e5, n), rng.uniform(2e4, 1e6, n), rng.uniform(0, 1e5, n),
                               rng.uniform(2e4, 2e6, n), rng.uniform(0, 6.28, n), 10e-6, liq)
    y = np.stack([rng.uniform(0.3, 3.0, n), rng.uniform(-2.0, 2.0, n)])
    tau = rng.uniform(0, 1, n)
    for k in range(2):
        v = np.zeros((2, n))
        v[k] = 1.0
        dt = oracle.rhs(oracle.KM_TAN, C, tau, np.vstack([y, v]))
        h = 1e-6 * np.maximum(np.abs(y[k]), 1.0)
        yp, ym = y.copy(), y.copy()
        yp[k] += h
        ym[k] -= h
        fd = (oracle.rhs(oracle.KM, C, tau, yp)[1] - oracle.rhs(oracle.KM, C, tau, ym)[1]) / (2 * h)
        scale = np.maximum(np.abs(fd), np.abs(oracle.rhs(oracle.KM, C, tau, y)[1]) / np.abs(y[k]).clip(1e-3))
        assert np.all(np.abs(dt[3] - fd) <= 1e-6 * scale + 1e-9), k
        # the state part is the plain right-hand side, the first tangent row v2
        np.testing.assert_array_equal(dt[:2], oracle.rhs(oracle.KM, C, tau, y))
        np.testing.assert_array_equal(dt[2], v[1])


def test_km_lyapunov_exponent_of_the_rest_state():
    """Unforced bubble at rest (P_A = 0, y = (1, 0)): the tangent equation is
    v' = J v with J the (constant) Jacobian there.  The per-phase log growths
    of the renormalised tangent vector add up to ln |exp(J k) v0| / |v0| after
    k phases (matrix exponential, J by central differences of the plain RHS):
    the renormalisation between phases loses nothing."""
    from scipy.linalg import expm
    liq = _liq(WATER_CFG)
    f = np.array([2e4, 1e5, 5e5])
    C = oracle.km_coefficients(0.0, f, 0.0, 0.0, 0.0, 10e-6, liq)
    y0 = np.vstack([np.ones(3), np.zeros(3), np.ones(3), np.ones(3)])
    tol = oracle.make_tol(rtol=1e-11, atol=1e-11, dt0=1e-2, dt_min=1e-14, dt_max=1e-1, n_phases=30,
                          phase_len=1.0, t0=0.0)
    r = oracle.cashkarp_solve(oracle.KM_TAN, C, y0, tol)
    assert np.all(r["status"] == 0) and r["acc"].shape[0] == 90
    growth = r["acc"][60:]                             # ln |v| per phase
    for j in range(3):
        J = np.zeros((2, 2))
        for k in range(2):
            yp = np.array([[1.0], [0.0]])
            ym = yp.copy()
            yp[k] += 1e-6
            ym[k] -= 1e-6
            Cj = C[:, j:j + 1]
            J[:, k] = (oracle.rhs(oracle.KM, Cj, 0.0, yp) - oracle.rhs(oracle.KM, Cj, 0.0, ym))[:, 0] / 2e-6
        lam = np.linalg.eigvals(J).real.max()
        assert lam < 0                                  # the rest state is stable
        v0 = np.array([1.0, 1.0]) / math.sqrt(2.0)
        exact = np.array([math.log(np.linalg.norm(expm(J * k) @ v0)) for k in range(1, 31)])
        np.testing.assert_allclose(np.cumsum(growth[:, j]), exact, rtol=1e-5, atol=1e-7)
        # once the transient of the non-normal J has passed, the per-phase growth
        # oscillates about lam (complex pair): the late mean is below zero
        assert growth[15:, j].mean() < 0


def test_km_dimensionless_form_equals_dimensional_equation():
    """y2' from C0..C12 equals R'' (2 pi / w1)^2 / R_E of the dimensional
    Keller-Miksis equation, including the dual-frequency terms."""
    rng = np.random.default_rng(11)
    liq = _liq(WATER_CFG)
    n = 200
    pA1 = rng.uniform(0.0, 2e5, n)
    pA2 = rng.uniform(0.0, 1e5, n)
    f1 = rng.uniform(2e4, 1e6, n)
    f2 = rng.uniform(1e4, 2e6, n)
    theta = rng.uniform(0.0, 2 * math.pi, n)
    RE = rng.uniform(2e-6, 50e-6, n)
    C = oracle.km_coefficients(pA1, f1, pA2, f2, theta, RE, liq)
    y1 = rng.uniform(0.3, 4.0, n)
    y2 = rng.uniform(-3.0, 3.0, n)
    tau = rng.uniform(0.0, 1.0, n)
    dy = oracle.rhs(oracle.KM, C, tau, np.stack([y1, y2]))
    assert np.array_equal(dy[0], y2)
    for i in range(n):
        w1 = 2 * math.pi * f1[i]
        R = y1[i] * RE[i]
        Rd = y2[i] * RE[i] * w1 / (2 * math.pi)
        t = tau[i] * 2 * math.pi / w1
        rdd = oracle.km_dimensional_rdd(R, Rd, t, pA1[i], f1[i], pA2[i], f2[i], theta[i], RE[i], liq)
        ref = rdd * (2 * math.pi / w1) ** 2 / RE[i]
        assert abs(dy[1, i] - ref) <= 1e-10 * max(1.0, abs(ref)), (i, dy[1, i], ref)


def test_km_small_amplitude_response_matches_linearisation():
    """For small P_A the radius follows the linearised equation about (1, 0),
    integrated here independently with SciPy; the gap is O(P_A^2)."""
    from scipy.integrate import solve_ivp

    liq = _liq(WATER_CFG)
    f = 1e5
    T = 3.0
    gaps = []
    for pA in (50.0, 100.0):
        C = oracle.km_coefficients(pA, f, 0.0, 0.0, 0.0, 10e-6, liq)[:, 0]
        # first-order Taylor expansion of N_KM / D_KM about y1 = 1, y2 = 0
        D0 = 1.0 + C[4] * C[9]
        kx = (C[3] - C[0] * C[10]) / D0
        kv = (C[1] - C[2] * C[9] - C[4]) / D0

        def lin(t, z):
            x, v = z
            force = -(C[5] * math.sin(2 * math.pi * t) + C[7] * math.cos(2 * math.pi * t)) / D0
            return [v, kx * x + kv * v + force]

        taus = np.linspace(0.25, T, 12)
        sol = solve_ivp(lin, (0.0, T), [0.0, 0.0], method="DOP853", rtol=1e-12, atol=1e-16,
                        t_eval=taus)
        x_nl = []
        for tt in taus:
            tol = oracle.make_tol(rtol=1e-12, atol=1e-14, dt0=1e-3, dt_min=1e-16, dt_max=1e-2,
                                  t0=0.0, t1=float(tt))
            r = oracle.cashkarp_solve(oracle.KM, C[:, None], [[1.0], [0.0]], tol)
            x_nl.append(r["y"][0, 0] - 1.0)
        x_nl = np.array(x_nl)
        amp = np.abs(sol.y[0]).max()
        assert amp > 0
        gaps.append(np.abs(x_nl - sol.y[0]).max() / amp)
    assert gaps[0] < 2e-3
    assert 1.6 < gaps[1] / gaps[0] < 2.5        # relative gap grows linearly in P_A


def test_km_function_evaluations_near_paper_table():
    """RHS evaluation counts at T = 1e-10 against the paper's MPGOS numbers
    (Table NumberFunctionEvaluation); the controller is unspecified there, so
    agreement within 15% is required, not equality."""
    g = json.load(open(os.path.join(GOLDEN, "km_function_evaluations.json")))
    liq = _liq(g["liquid"])
    f = np.array(g["f1_Hz"])
    C = oracle.km_coefficients(g["pA1_Pa"], f, 0.0, 0.0, 0.0, g["RE_m"], liq)
    tol = oracle.make_tol(rtol=g["tol"], atol=g["tol"], dt0=1e-2, dt_min=1e-14, dt_max=1e-1,
                          t0=0.0, t1=g["tau_end"])
    r = oracle.cashkarp_solve(oracle.KM, C, np.stack([np.ones(3), np.zeros(3)]), tol)
    ratio = r["nrhs"] / np.array(g["nf_mpgos"])
    assert np.all(np.abs(ratio - 1.0) < 0.15), ratio


def test_km_dopri5_function_evaluations_near_paper_table():
    """The same runs with the Dormand-Prince pair against the paper's Julia
    column (DifferentialEquations.jl uses Dormand-Prince there); its
    controller differs from this one, so 10% is required, not equality."""
    g = json.load(open(os.path.join(GOLDEN, "km_function_evaluations.json")))
    liq = _liq(g["liquid"])
    f = np.array(g["f1_Hz"])
    C = oracle.km_coefficients(g["pA1_Pa"], f, 0.0, 0.0, 0.0, g["RE_m"], liq)
    tol = oracle.make_tol(rtol=g["tol"], atol=g["tol"], dt0=1e-2, dt_min=1e-14, dt_max=1e-1,
                          t0=0.0, t1=g["tau_end"], method=oracle.DOPRI5)
    r = oracle.cashkarp_solve(oracle.KM, C, np.stack([np.ones(3), np.zeros(3)]), tol)
    ratio = r["nrhs"] / np.array(g["nf_julia_dopri5"])
    assert np.all(np.abs(ratio - 1.0) < 0.10), ratio
    # and the Cash-Karp run needs fewer evaluations than Dormand-Prince (the
    # table's N_F^M / N_F^J < 1 at every frequency)
    tol.method = oracle.CASHKARP
    rc = oracle.cashkarp_solve(oracle.KM, C, np.stack([np.ones(3), np.zeros(3)]), tol)
    assert np.all(rc["nrhs"] < r["nrhs"])


def _nf_at_global_error(method, target=1e-10):
    """N_F at global error E = target, interpolated log-log between the two
    tolerances T = 10^-k that bracket it (the paper reads its table off the
    N_F(E) curves; the reference solution is the T = 1e-15 run)."""
    g = json.load(open(os.path.join(GOLDEN, "km_function_evaluations.json")))
    liq = _liq(g["liquid"])
    f = np.array(g["f1_Hz"])
    C = oracle.km_coefficients(g["pA1_Pa"], f, 0.0, 0.0, 0.0, g["RE_m"], liq)
    y0 = np.stack([np.ones(3), np.zeros(3)])
    runs = {}
    for k in range(8, 16):
        tol = oracle.make_tol(rtol=10.0 ** -k, atol=10.0 ** -k, dt0=1e-2, dt_min=1e-14, dt_max=1e-1,
                              t0=0.0, t1=g["tau_end"], method=method)
        r = oracle.cashkarp_solve(oracle.KM, C, y0, tol)
        runs[k] = (r["y"][0], r["nrhs"].astype(float))
    ref = runs[15][0]
    out = []
    for j in range(3):
        E = {k: abs(runs[k][0][j] - ref[j]) for k in range(8, 15)}
        for k in range(8, 14):
            if E[k] >= target > E[k + 1]:
                w = np.log(E[k] / target) / np.log(E[k] / E[k + 1])
                out.append(runs[k][1][j] ** (1 - w) * runs[k + 1][1][j] ** w)
                break
        else:
            out.append(np.nan)
    return np.array(out), g["global_error_1e-10"]


def test_nf_at_global_error_near_paper_table():
    """Work for a global error of 1e-10 (Table NumberFunctionEvaluationGlobalError):
    Dormand-Prince against the Julia column within 10%, Cash-Karp against the
    MPGOS column within 25% (its 20 kHz entry sits where the N_F(E) curve
    bends; our controller is not the paper's)."""
    dp, g = _nf_at_global_error(oracle.DOPRI5)
    ck, _ = _nf_at_global_error(oracle.CASHKARP)
    assert np.all(np.abs(dp / np.array(g["nf_julia_dopri5"]) - 1) < 0.10), dp
    assert np.all(np.abs(ck / np.array(g["nf_mpgos"]) - 1) < 0.25), ck


def test_km_global_error_tracks_tolerance():
    """E = |y1(2) - y1^E(2)| against a T = 1e-15 run (Sec. 4.2.2 method)."""
    g = json.load(open(os.path.join(GOLDEN, "km_function_evaluations.json")))
    liq = _liq(g["liquid"])
    f = np.array(g["f1_Hz"])
    C = oracle.km_coefficients(g["pA1_Pa"], f, 0.0, 0.0, 0.0, g["RE_m"], liq)
    y0 = np.stack([np.ones(3), np.zeros(3)])

    def run(tv):
        tol = oracle.make_tol(rtol=tv, atol=tv, dt0=1e-2, dt_min=1e-16, dt_max=1e-1, t0=0.0, t1=2.0)
        return oracle.cashkarp_solve(oracle.KM, C, y0, tol)["y"][0]

    ref = run(1e-15)
    e_prev = None
    for tv in (1e-12, 1e-10, 1e-8):
        e = np.abs(run(tv) - ref)
        assert np.all(e < 30 * tv), (tv, e)
        if e_prev is not None:
            assert np.all(e > e_prev)
        e_prev = e


# ---------------------------------------------------------------------------
# pressure relief valve (Sec. 4.3) and the event machinery
# ---------------------------------------------------------------------------

PRV = dict(kappa=1.25, delta=10.0, beta=20.0, r=0.8)


def _prv_params(q):
    q = np.atleast_1d(np.asarray(q, dtype=float))
    one = np.ones_like(q)
    return np.stack([q, PRV["kappa"] * one, PRV["delta"] * one, PRV["beta"] * one, PRV["r"] * one])


def _prv_tol(t1=1024.0, acc_t_start=512.0):
    return oracle.make_tol(rtol=1e-10, atol=1e-10, dt0=1e-3, dt_min=1e-14, dt_max=1.0,
                           event_tol=1e-6, t0=0.0, t1=t1, acc_t_start=acc_t_start)


def test_prv_equilibrium_is_stationary():
    """y1*^2 (y1* + delta) = q^2, y2 = 0, y3 = y1* + delta is a fixed point."""
    for q in (0.5, 3.0, 9.0):
        roots = np.roots([1.0, PRV["delta"], 0.0, -q * q])
        y1s = float(max(r.real for r in roots if abs(r.imag) < 1e-12))
        yeq = np.array([[y1s], [0.0], [y1s + PRV["delta"]]])
        dy = oracle.rhs(oracle.PRV, _prv_params(q), 0.0, yeq)
        assert np.abs(dy).max() < 1e-12 * 20


def test_prv_bifurcation_impacting_range():
    """The valve hits the seat (min y1 = 0) for q up to about 7.5 and not
    beyond (Sec. 4.3, bifurcation diagram)."""
    q = np.array([0.3, 1.0, 3.0, 5.0, 7.0, 8.5, 9.5])
    n = q.size
    y0 = np.stack([np.full(n, 0.2), np.zeros(n), np.zeros(n)])
    r = oracle.cashkarp_solve(oracle.PRV, _prv_params(q), y0, _prv_tol(), nthreads=0)
    assert np.all(r["status"] == 0)
    ymin = r["acc"][32]
    nimp = r["acc"][34]
    impacting = q < 7.5
    assert np.all(ymin[impacting] == 0.0)
    assert np.all(nimp[impacting] > 10)
    assert np.all(ymin[~impacting] > 0.05)
    assert np.all(r["y"][2] >= 0.0)
    assert np.all(r["t"] == 1024.0)


def test_bouncing_ball_event_location_and_impact_law():
    """Ball: y1'' = -g, impact y2+ = -r y2-.  Apex heights after k bounces are
    r^(2k) h0 and the k-th impact time is sqrt(2h0/g)(1 + 2 sum_{j<k} r^j)."""
    g, rr, h0 = 1.0, 0.8, 1.0
    T = 10.0
    tol = oracle.make_tol(rtol=1e-10, atol=1e-10, dt0=1e-3, dt_min=1e-14, dt_max=1.0,
                          event_tol=1e-6, t0=0.0, t1=T, acc_t_start=0.0)
    r = oracle.cashkarp_solve(oracle.BALL, [[g], [rr]], [[h0], [0.0], [0.0]], tol)
    assert r["status"][0] == 0
    t_imp = [math.sqrt(2 * h0 / g)]
    while True:
        k = len(t_imp)
        nxt = t_imp[-1] + 2 * rr ** k * math.sqrt(2 * h0 / g)
        if nxt > T:
            break
        t_imp.append(nxt)
    n_imp = int(r["acc"][34, 0])
    n_max = int(r["acc"][33, 0])
    assert n_imp == len(t_imp)
    # apexes between impacts (the start apex at t = 0 is not a crossing)
    assert n_max in (n_imp - 1, n_imp)
    for m in range(min(n_max, oracle.RING)):
        h = r["acc"][m, 0]
        assert abs(h - rr ** (2 * (m + 1)) * h0) < 1e-5 * h0, (m, h)
    assert r["acc"][32, 0] == 0.0           # it touched the floor


def test_grazing_impact_is_located_at_the_closed_form_root():
    """Ball with upward acceleration (g < 0) approaching the floor: y1 = h0 +
    v0 t - g t^2 / 2 dips 1.2e-5 below the seat, far less than the step, a
    grazing impact.  The first crossing is t* = (-v0 - sqrt(v0^2 - 2 |g| h0))
    / |g|; after the impact law y2 <- -r y2 the flight is again a parabola, so
    y1(T) has a closed form.  Cash-Karp integrates the quadratic exactly, so
    only the event location separates the solver from it."""
    g, rr, h0, v0 = -36.14, 0.8, 0.00137, -0.316
    a = -g
    ts = (-v0 - math.sqrt(v0 * v0 - 2.0 * a * h0)) / a
    vs = v0 + a * ts
    T = 0.02
    vp = -rr * vs
    y_T = vp * (T - ts) + 0.5 * a * (T - ts) ** 2
    tol = oracle.make_tol(rtol=1e-10, atol=1e-10, dt0=0.0089, dt_min=1e-14, dt_max=1.0,
                          event_tol=1e-6, t0=0.0, t1=T, acc_t_start=0.0)
    r = oracle.cashkarp_solve(oracle.BALL, [[g], [rr]], [[h0], [v0], [0.0]], tol)
    assert r["status"][0] == 0
    assert int(r["acc"][34, 0]) == 1
    assert abs(r["y"][0, 0] - y_T) < 1e-9, (r["y"][0, 0], y_T)
    assert r["nrej"][0] + r["nacc"][0] < 40


def test_prv_grazing_impact_from_a_recorded_state():
    """A valve state near the edge of the impacting range (q = 7.5393) that
    approaches the seat at y2 = -0.316 under a strong opening force and dips
    about 1e-5 below it: the impact must be located (status 0, one impact)."""
    q = 7.5392987796736906
    y0 = np.array([[0.0013698420381308958], [-0.3162497537150412], [45.746744783524875]])
    tol = oracle.make_tol(rtol=1e-10, atol=1e-10, dt0=0.008889370476683223, dt_min=1e-14, dt_max=1.0,
                          event_tol=1e-6, t0=0.0, t1=0.05, acc_t_start=0.0)
    r = oracle.cashkarp_solve(oracle.PRV, _prv_params(q), y0, tol)
    assert r["status"][0] == 0
    assert int(r["acc"][34, 0]) == 1
    assert r["acc"][32, 0] == 0.0


def test_prv_sticking_interval_has_the_closed_form():
    """Sticking (a reading; the paper is silent): after an impact whose
    rebound cannot leave the event band, the valve rests on the seat
    (y1 = y2 = 0) and y3' = beta q exactly, until y3 reaches delta at
    t_lift = t + (delta - y3) / (beta q).

    The valve starts on the seat with y3 = 5 < delta: the seat force pushes it
    down, the first step is cut back to an impact with a tiny rebound, and it
    sticks.  Before t_lift = (delta - 5) / (beta q) = 0.25 the state must be
    (0, 0, 5 + beta q t).  After it, the valve leaves the seat from
    (0, 0, delta) at rest, and the Taylor series of Eqs.
    pressure_relief_valve_1-3 about that point, with s = t - t_lift, is
      y1 = beta q s^3/6 - kappa beta q s^4/24 + beta q (kappa^2 - 1) s^5/120
           + (beta q (2 kappa - kappa^3) - beta^2 q sqrt(delta)) s^6/720 + O(s^7),
      y3 = delta + beta q s - beta^2 q sqrt(delta) s^4/24 + O(s^5).
    A lift time off by d moves y1(s) by about 3 d / s relative, so the
    2e-7 bound below catches d > 1e-9; a wrong sign or rate in the closed
    form fails outright.  (The short motion before the valve sticks, with
    y1 slightly below zero, raises y3 by 4.7e-9 more than beta q t, so the
    lift comes 2.3e-10 early: 1.4e-7 of y1 at s = 0.005.)"""
    q, kappa, delta, beta, rr = 1.0, 1.25, 10.0, 20.0, 0.8
    P = _prv_params(q)
    y30 = 5.0
    t_lift = (delta - y30) / (beta * q)
    for t1 in (0.1, t_lift - 1e-3):
        tol = oracle.make_tol(rtol=1e-10, atol=1e-10, dt0=1e-3, dt_min=1e-14, dt_max=1.0, event_tol=1e-6,
                              t0=0.0, t1=t1, acc_t_start=0.0)
        r = oracle.cashkarp_solve(oracle.PRV, P, [[0.0], [0.0], [y30]], tol)
        assert r["status"][0] == 0 and r["t"][0] == t1
        assert r["y"][0, 0] == 0.0 and r["y"][1, 0] == 0.0
        assert int(r["acc"][34, 0]) == 1                     # the one impact that made it stick
        # the impact took about 5e-4 of time with |y1| < 1e-6, so y3 followed beta q
        # to within beta * 1e-6 * sqrt(delta) * 5e-4 < 1e-7
        assert abs(r["y"][2, 0] - (y30 + beta * q * t1)) < 1e-7
    for s in (0.005, 0.01, 0.02):
        tol = oracle.make_tol(rtol=1e-12, atol=1e-12, dt0=1e-3, dt_min=1e-14, dt_max=1.0, event_tol=1e-6,
                              t0=0.0, t1=t_lift + s, acc_t_start=0.0)
        r = oracle.cashkarp_solve(oracle.PRV, P, [[0.0], [0.0], [y30]], tol)
        assert r["status"][0] == 0
        bq = beta * q
        y1 = (bq * s ** 3 / 6 - kappa * bq * s ** 4 / 24 + bq * (kappa ** 2 - 1) * s ** 5 / 120
              + (bq * (2 * kappa - kappa ** 3) - beta ** 2 * q * math.sqrt(delta)) * s ** 6 / 720)
        y3 = delta + bq * s - beta ** 2 * q * math.sqrt(delta) * s ** 4 / 24
        assert abs(r["y"][0, 0] / y1 - 1.0) < 2e-7, (s, r["y"][0, 0], y1)
        assert abs(r["y"][2, 0] - y3) < 1e-8 * delta, (s, r["y"][2, 0], y3)
        assert int(r["acc"][34, 0]) == 1


def test_prv_impacts_keep_body_on_or_above_seat():
    q = np.array([0.5, 2.0, 6.0])
    y0 = np.stack([np.full(3, 0.2), np.zeros(3), np.zeros(3)])
    r = oracle.cashkarp_solve(oracle.PRV, _prv_params(q), y0, _prv_tol(t1=200.0, acc_t_start=0.0))
    assert np.all(r["acc"][32] >= -1e-6)     # within the event tolerance
