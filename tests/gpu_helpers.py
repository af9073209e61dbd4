"""Helpers of the GPU parity tests: run a workload through the C ABI and the
same workload through the oracle, and the conditioning-aware comparison."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2011_01740_gb300 as ens
from paper_2011_01740_gb300 import workloads as W

EPS = 2.0 ** -52

ORACLE_SYS = {ens.ENS_SYS_TOY_X2P: oracle.X2P, ens.ENS_SYS_LORENZ: oracle.LORENZ,
              ens.ENS_SYS_KELLER_MIKSIS: oracle.KM, ens.ENS_SYS_RELIEF_VALVE: oracle.PRV}


def solve_gpu(sys, params, y0, t_span, solver, tol, launch=None, stream=None, reads=None):
    """Create, solve, read every output, destroy.  Returns a dict of numpy arrays."""
    n = params.shape[1] if hasattr(params, "shape") else len(params[0])
    ctx = ens.ens_create(sys, n, params, y0, t_span, solver, tol)
    try:
        if launch is not None:
            ens.ens_set_launch(ctx, launch)
        ens.ens_solve(ctx, stream)
        sync = ens.ens_sync(ctx)
        sel = reads or (ens.ENS_STATE, ens.ENS_ACC, ens.ENS_STATUS, ens.ENS_NSTEPS, ens.ENS_NREJ,
                        ens.ENS_NRHS, ens.ENS_TIME, ens.ENS_DT)
        out = {"sync": sync}
        names = {ens.ENS_STATE: "y", ens.ENS_ACC: "acc", ens.ENS_STATUS: "status",
                 ens.ENS_NSTEPS: "nacc", ens.ENS_NREJ: "nrej", ens.ENS_NRHS: "nrhs",
                 ens.ENS_TIME: "t", ens.ENS_DT: "dt"}
        for w in sel:
            if w == ens.ENS_ACC and ens.ens_acc_rows(ctx) == 0:
                out["acc"] = np.zeros((0, n))
                continue
            out[names[w]] = ens.ens_read(ctx, w)
        out["launch"] = ens.ens_get_launch(ctx).as_dict()
        return out
    finally:
        ens.ens_destroy(ctx)


def ens_tol_from(t: W.Tolerances, **kw):
    d = dict(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
             event_tol=t.event_tol, max_steps=t.max_steps, n_phases=t.n_phases,
             phase_len=t.phase_len, acc_t_start=t.acc_t_start)
    d.update(kw)
    return ens.make_tol(**d)


def oracle_tol_from(t: W.Tolerances, **kw):
    d = dict(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
             event_tol=t.event_tol, max_steps=t.max_steps, n_phases=t.n_phases,
             phase_len=t.phase_len, t0=t.t0, t1=t.t1, acc_t_start=t.acc_t_start)
    d.update(kw)
    return oracle.make_tol(**d)


def km_coeffs_oracle(phys, liquid):
    return oracle.km_coefficients(phys["pA1"], phys["f1"], phys["pA2"], phys["f2"], phys["theta"],
                                  phys["RE"], oracle.liquid(**liquid))


def km_coeffs_lib(phys, liquid):
    return ens.ens_km_coefficients(phys["pA1"], phys["f1"], phys["pA2"], phys["f2"], phys["theta"],
                                   phys["RE"], liquid)


def rel_err(a, b, axis=0):
    """Per-system max-norm relative error ||a - b||_inf / max(||b||_inf, 1e-300)."""
    d = np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))
    d = np.where(np.isnan(d) & np.isnan(b) & np.isnan(a), 0.0, d)
    return d.max(axis) / np.maximum(np.nanmax(np.abs(b), axis), 1e-300)


def rk4_amplification(sys, params, y0, dt, nsteps, delta=1e-10):
    """Growth factor of a relative perturbation of the initial state over the
    run, from two oracle solves: A = |y(y0 (1 + delta)) - y(y0)| / (delta |y|)."""
    a, _ = oracle.rk4_solve(ORACLE_SYS[sys], params, y0, 0.0, dt, nsteps)
    b, _ = oracle.rk4_solve(ORACLE_SYS[sys], params, np.asarray(y0) * (1 + delta), 0.0, dt, nsteps)
    return a, np.maximum(rel_err(b, a) / delta, 1.0)


def rk4_tolerance(amplification, nsteps=1000):
    """Fixed-step FP64 bound: 1e-12 relative, widened where rounding
    accumulates.  A contracted (FMA) kernel and the uncontracted oracle differ
    by O(eps) at every operation of every step; a difference made at step j
    grows by at most the amplification A of the run, so after N steps the gap
    is at most about c N eps A with c the operations per state component and
    step (c = 8 here; the measured worst case over the Lorenz sweep is
    258 eps A with N = 1000)."""
    return np.maximum(1e-12, 8 * nsteps * EPS * amplification)
