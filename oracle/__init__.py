"""CPU oracle for the ensemble ODE method of arXiv 2011.01740 (test infrastructure).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2011_01740_gb300``) never touches it, and
this package imports nothing from the product path.

The arithmetic lives in ``oracle.c`` (plain C, IEEE double, no FMA
contraction, libm); this module builds it with gcc and marshals numpy arrays
through ctypes.  ``mlp.py`` holds the float64 numpy reference of the surrogate
network.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, exact quadrature/order conditions, an
independent dimensional route, or numbers printed in the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# system identifiers (mirror the enum in oracle.c)
X2P, LORENZ, KM, PRV, LINEAR, TPOW, BALL, KM_TAN, FCOS = range(9)
CASHKARP, DOPRI5 = 0, 1                     # Tol.method
DIM = {X2P: 1, LORENZ: 3, KM: 2, PRV: 3, LINEAR: 1, TPOW: 1, BALL: 3, KM_TAN: 4, FCOS: 1}
NPAR = {X2P: 1, LORENZ: 3, KM: 13, PRV: 5, LINEAR: 1, TPOW: 2, BALL: 2, KM_TAN: 13, FCOS: 1}

ST_DT_UNDERFLOW, ST_MAX_STEPS, ST_NONFINITE, ST_EVENT_NO_CONVERGE = 1, 2, 4, 8
RING = 32


class Liquid(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("c", ctypes.c_double), ("mu", ctypes.c_double),
                ("sigma", ctypes.c_double), ("pv", ctypes.c_double), ("pinf", ctypes.c_double),
                ("gamma", ctypes.c_double)]


class Tol(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("dt0", ctypes.c_double), ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("event_tol", ctypes.c_double), ("max_steps", ctypes.c_int64),
                ("n_phases", ctypes.c_int32), ("phase_len", ctypes.c_double),
                ("t0", ctypes.c_double), ("t1", ctypes.c_double),
                ("acc_t_start", ctypes.c_double), ("method", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FMA contraction, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.orc_rhs.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, dp, dp]
        L.orc_km_coefficients.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, dp,
                                          ctypes.POINTER(Liquid), dp]
        L.orc_km_dimensional_rdd.argtypes = [ctypes.c_double] * 9 + [ctypes.POINTER(Liquid)]
        L.orc_km_dimensional_rdd.restype = ctypes.c_double
        L.orc_rk4_step.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_rk4_solve.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int64, i32p, ctypes.c_int]
        L.orc_cashkarp_tableau.argtypes = [dp, dp, dp, dp]
        L.orc_dopri5_tableau.argtypes = [dp, dp, dp, dp]
        L.orc_dopri5_step.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
        L.orc_cashkarp_step.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp,
                                        dp, dp]
        L.orc_cashkarp_solve.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp,
                                         ctypes.POINTER(Tol), dp, dp, dp, i32p, i64p, i64p, i64p,
                                         ctypes.c_int]
        L.orc_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---------------------------------------------------------------------------
# liquids
# ---------------------------------------------------------------------------

def liquid(rho, c, mu, sigma, pv, pinf, gamma) -> Liquid:
    return Liquid(rho, c, mu, sigma, pv, pinf, gamma)


# ---------------------------------------------------------------------------
# right-hand sides, coefficients
# ---------------------------------------------------------------------------

def rhs(sys: int, params, t, y):
    """One RHS evaluation per system; params (npar, n), t (n,), y (dim, n)."""
    params = _c64(params).reshape(NPAR[sys], -1)
    n = params.shape[1]
    y = _c64(y).reshape(DIM[sys], n)
    t = _c64(np.broadcast_to(np.asarray(t, dtype=np.float64), (n,)))
    dy = np.empty_like(y)
    lib().orc_rhs(sys, n, _d(params), _d(t), _d(y), _d(dy))
    return dy


def km_coefficients(pA1, f1, pA2, f2, theta, RE, liq: Liquid):
    """C0..C12 per system (13, n) from SI physical parameters (Eq. coefficients)."""
    arrs = np.broadcast_arrays(*[np.asarray(a, dtype=np.float64) for a in (pA1, f1, pA2, f2, theta, RE)])
    arrs = [_c64(a).ravel() for a in arrs]
    n = arrs[0].size
    out = np.empty((13, n), dtype=np.float64)
    lib().orc_km_coefficients(n, *[_d(a) for a in arrs], ctypes.byref(liq), _d(out))
    return out


def km_dimensional_rdd(R, Rd, t, pA1, f1, pA2, f2, theta, RE, liq: Liquid) -> float:
    """R'' (m/s^2) from the dimensional Keller-Miksis equation (Eqs. keller_miksis_1-4)."""
    return float(lib().orc_km_dimensional_rdd(R, Rd, t, pA1, f1, pA2, f2, theta, RE,
                                              ctypes.byref(liq)))


# ---------------------------------------------------------------------------
# RK4
# ---------------------------------------------------------------------------

def rk4_step(sys: int, p, t: float, h: float, y):
    p = _c64(p)
    y = _c64(y)
    out = np.empty(DIM[sys])
    lib().orc_rk4_step(sys, _d(p), t, h, _d(y), _d(out))
    return out


def rk4_solve(sys: int, params, y0, t0: float, dt: float, nsteps: int, nthreads: int = 0):
    """Fixed-step RK4 of every system; returns (y (dim, n), status (n,))."""
    params = _c64(params).reshape(NPAR[sys], -1)
    n = params.shape[1]
    y = _c64(y0).reshape(DIM[sys], n).copy()
    status = np.zeros(n, dtype=np.int32)
    lib().orc_rk4_solve(sys, n, _d(params), _d(y), t0, dt, nsteps,
                        status.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), nthreads)
    return y, status


# ---------------------------------------------------------------------------
# Cash-Karp
# ---------------------------------------------------------------------------

def cashkarp_tableau():
    c = np.empty(6)
    a = np.empty(36)
    b = np.empty(6)
    bs = np.empty(6)
    lib().orc_cashkarp_tableau(_d(c), _d(a), _d(b), _d(bs))
    return c, a.reshape(6, 6), b, bs


def dopri5_tableau():
    c = np.empty(7)
    a = np.empty(49)
    b = np.empty(7)
    bs = np.empty(7)
    lib().orc_dopri5_tableau(_d(c), _d(a), _d(b), _d(bs))
    return c, a.reshape(7, 7), b, bs


def dopri5_step(sys: int, p, t: float, h: float, y):
    p = _c64(p)
    y = _c64(y)
    y5 = np.empty(DIM[sys])
    err = np.empty(DIM[sys])
    lib().orc_dopri5_step(sys, _d(p), t, h, _d(y), _d(y5), _d(err))
    return y5, err


def cashkarp_step(sys: int, p, t: float, h: float, y):
    p = _c64(p)
    y = _c64(y)
    y5 = np.empty(DIM[sys])
    err = np.empty(DIM[sys])
    lib().orc_cashkarp_step(sys, _d(p), t, h, _d(y), _d(y5), _d(err))
    return y5, err


def make_tol(rtol=1e-10, atol=1e-10, dt0=1e-2, dt_min=1e-14, dt_max=1e-1, event_tol=1e-6,
             max_steps=10**9, n_phases=0, phase_len=1.0, t0=0.0, t1=1.0,
             acc_t_start=0.0, method=0) -> Tol:
    """method: CASHKARP (0) or DOPRI5 (1)."""
    return Tol(rtol, atol, dt0, dt_min, dt_max, event_tol, int(max_steps), int(n_phases),
               phase_len, t0, t1, acc_t_start, int(method))


def n_acc_rows(sys: int, tol: Tol) -> int:
    if tol.n_phases > 0:
        return (3 if sys == KM_TAN else 2) * tol.n_phases
    if sys in (PRV, BALL):
        return RING + 3
    return 0


def cashkarp_solve(sys: int, params, y0, tol: Tol, nthreads: int = 0):
    """Adaptive Cash-Karp solve of every system (phase / event / plain mode).

    Returns a dict with y (dim, n), t, dt, acc (rows, n), status, nacc, nrej, nrhs.
    """
    params = _c64(params).reshape(NPAR[sys], -1)
    n = params.shape[1]
    y = _c64(y0).reshape(DIM[sys], n).copy()
    rows = n_acc_rows(sys, tol)
    acc = np.empty((max(rows, 1), n))
    t = np.empty(n)
    dt = np.empty(n)
    status = np.zeros(n, dtype=np.int32)
    nacc = np.zeros(n, dtype=np.int64)
    nrej = np.zeros(n, dtype=np.int64)
    nrhs = np.zeros(n, dtype=np.int64)
    i32 = ctypes.POINTER(ctypes.c_int32)
    i64 = ctypes.POINTER(ctypes.c_int64)
    lib().orc_cashkarp_solve(sys, n, _d(params), _d(y), ctypes.byref(tol), _d(t), _d(dt),
                             _d(acc) if rows else None, status.ctypes.data_as(i32),
                             nacc.ctypes.data_as(i64), nrej.ctypes.data_as(i64),
                             nrhs.ctypes.data_as(i64), nthreads)
    return {"y": y, "t": t, "dt": dt, "acc": acc[:rows], "status": status, "nacc": nacc,
            "nrej": nrej, "nrhs": nrhs}
