"""GPU parity of the Dormand-Prince 5(4) pair (ENS_DOPRI5; the solver of the
paper's Julia runs, Sec. 4.2) against the oracle's Dormand-Prince solve:
Keller-Miksis phase mode, the relief valve with events, the plain mode, the
first-same-as-last evaluation count and launch-shape invariance.

Comparisons run on the well-conditioned systems, where the GPU must match to
1e-8 relative, as for Cash-Karp.  Well-conditioned means the oracle's
accessories move by less than 1e-9 under 1e-14 relative perturbations of the
initial state and under a 1e-12 relative change of the first step, which
shifts the whole step sequence (rounding differences between the two sides
do the same): some impacting valves move by 5e-8 under the latter alone.
"""
import numpy as np
import pytest

import oracle
import paper_2011_01740_gb300 as ens
from paper_2011_01740_gb300 import workloads as W
from gpu_helpers import ens_tol_from, km_coeffs_lib, km_coeffs_oracle, oracle_tol_from, rel_err, solve_gpu

pytestmark = pytest.mark.gpu

ACC_TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ens.lib()


def _oracle_dp(sys, params, y0, otol, rows=slice(None)):
    """Oracle run plus its well-conditioned subset, judged on acc[rows] (the
    value rows; the relief valve's event counts, rows 33 and 34, must not
    move at all)."""
    a = oracle.cashkarp_solve(sys, params, y0, otol)
    shifted = oracle.make_tol(**{f: getattr(otol, f) for f, _ in otol._fields_})
    shifted.dt0 = otol.dt0 * (1 + 1e-12)
    runs = [oracle.cashkarp_solve(sys, params, np.asarray(y0) * (1 + d), otol) for d in (1e-14, -3e-15)]
    runs.append(oracle.cashkarp_solve(sys, params, y0, shifted))
    well = a["status"] == 0
    for b in runs:
        well &= (rel_err(b["acc"][rows], a["acc"][rows]) < 1e-9) & (b["status"] == 0)
        if sys == oracle.PRV:
            well &= np.all(b["acc"][33:35] == a["acc"][33:35], axis=0)
    return a, well


def _km(km, launch=None, **kw):
    C = km_coeffs_lib(km["phys"], km["liquid"])
    t = km["tol"]
    return solve_gpu(ens.ENS_SYS_KELLER_MIKSIS, C, km["y0"], (t.t0, t.t1), ens.ENS_DOPRI5,
                     ens_tol_from(t, **kw), launch=launch)


def test_km_phase_mode_parity():
    km = W.km(19, 23, n_phases=4)          # 437 systems: several blocks and a ragged tail
    g = _km(km)
    Co = km_coeffs_oracle(km["phys"], km["liquid"])
    r, well = _oracle_dp(oracle.KM, Co, km["y0"], oracle_tol_from(km["tol"], method=oracle.DOPRI5))
    assert g["sync"] == ens.ENS_OK and np.all(g["status"] == 0)
    assert well.mean() > 0.9
    err = rel_err(g["acc"], r["acc"])
    assert np.all(err[well] < ACC_TOL), err[well].max()
    d = np.abs(g["nacc"] - r["nacc"]) / r["nacc"]
    assert np.median(d[well]) == 0.0 and d[well].max() <= 0.05
    # first same as last: one fresh k1 per phase start, 6 evaluations per trial
    assert np.all(g["nrhs"] == 4 + 6 * (g["nacc"] + g["nrej"]))


def test_km_dopri5_needs_more_evaluations_than_cash_karp():
    """The paper's Table NumberFunctionEvaluation: the Dormand-Prince runs
    need more right-hand-side evaluations than Cash-Karp at T = 1e-10."""
    km = W.km(9, 12, n_phases=2)
    C = km_coeffs_lib(km["phys"], km["liquid"])
    t = km["tol"]
    ck = solve_gpu(ens.ENS_SYS_KELLER_MIKSIS, C, km["y0"], (t.t0, t.t1), ens.ENS_RKCK45, ens_tol_from(t))
    dp = _km(km)
    forced = km["phys"]["pA1"] > 0
    assert dp["nrhs"][forced].sum() > ck["nrhs"][forced].sum()


def test_relief_valve_events_parity():
    wl = W.prv(300, t1=64.0)
    t = wl["tol"]
    g = solve_gpu(ens.ENS_SYS_RELIEF_VALVE, wl["params"], wl["y0"], (t.t0, t.t1), ens.ENS_DOPRI5,
                  ens_tol_from(t))
    r, well = _oracle_dp(oracle.PRV, wl["params"], wl["y0"], oracle_tol_from(t, method=oracle.DOPRI5),
                         rows=slice(0, 33))
    assert g["sync"] == ens.ENS_OK and np.all(g["status"] == 0)
    assert well.mean() > 0.75, well.mean()
    acc = g["acc"]
    assert np.array_equal(acc[33][well], r["acc"][33][well])     # maxima
    assert np.array_equal(acc[34][well], r["acc"][34][well])     # impacts
    assert np.all(rel_err(acc[:33], r["acc"][:33])[well] < ACC_TOL)
    assert np.all(rel_err(g["y"], r["y"])[well] < 1e-7)


def test_plain_mode_lorenz_parity():
    """Plain adaptive integration over [0, 2] (no phases, no events)."""
    n = 200
    rho = np.linspace(0.0, 21.0, n)
    params = np.stack([rho, np.full(n, 10.0), np.full(n, 8.0 / 3.0)])
    y0 = np.full((3, n), 10.0)
    kw = dict(rtol=1e-10, atol=1e-10, dt0=1e-3, dt_min=1e-14, dt_max=0.1)
    g = solve_gpu(ens.ENS_SYS_LORENZ, params, y0, (0.0, 2.0), ens.ENS_DOPRI5, ens.make_tol(**kw))
    r = oracle.cashkarp_solve(oracle.LORENZ, params, y0,
                              oracle.make_tol(t0=0.0, t1=2.0, method=oracle.DOPRI5, **kw))
    assert g["sync"] == ens.ENS_OK and np.all(g["t"] == 2.0)
    assert np.all(rel_err(g["y"], r["y"]) < 1e-8)
    assert np.all(g["nrhs"] == 1 + 6 * (g["nacc"] + g["nrej"]))


def test_launch_shapes_are_bitwise_identical():
    km = W.km(60, 50, n_phases=2)          # 3,000 systems
    ref = _km(km, launch=ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=128))
    for L in (ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=160, blocks_per_sm=1, cost_order=1,
                              use_graph=1),
              ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=32, blocks_per_sm=1, cost_order=0)):
        g = _km(km, launch=L)
        for k in ("y", "acc", "nacc", "nrej", "nrhs", "status", "dt"):
            assert np.array_equal(g[k], ref[k], equal_nan=True), (k, L.as_dict())


def test_fp32_variant_is_cash_karp_only():
    km = W.km(2, 2, n_phases=1)
    C = km_coeffs_lib(km["phys"], km["liquid"])
    with pytest.raises(ens.EnsError) as e:
        ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0), ens.ENS_DOPRI5,
                       ens.make_tol(n_phases=1, prec=ens.ENS_FP32_COMP, rtol=1e-8, atol=1e-8))
    assert e.value.status == ens.ENS_ENOTSUP
