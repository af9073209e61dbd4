"""Right-hand-side parity on random states: the device functions the solvers
inline (through ens_eval_rhs) against the oracle's plain evaluation."""
import numpy as np
import pytest

import oracle
import paper_2011_01740_gb300 as ens
from paper_2011_01740_gb300 import workloads as W
from gpu_helpers import km_coeffs_oracle

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _eval(sys, params, t, y):
    import torch
    n = t.size
    dy = torch.empty(y.shape, dtype=torch.float64, device="cuda")
    ens.ens_eval_rhs(sys, n, _dev(params), _dev(t), _dev(y), dy)
    torch.cuda.synchronize()
    return dy.cpu().numpy()


@pytest.mark.parametrize("dual", [False, True])
def test_keller_miksis_rhs(dual):
    """Random states and drivings, including quadrant boundaries of the
    forcing phase; error measured against the magnitude of the terms that
    cancel in N_KM."""
    rng = np.random.default_rng(21 + dual)
    n = 20000
    phys = dict(pA1=rng.uniform(0, 2e5, n), f1=np.exp(rng.uniform(np.log(2e4), np.log(1e6), n)),
                pA2=rng.uniform(0, 1e5, n) if dual else np.zeros(n),
                f2=rng.uniform(1e4, 2e6, n) if dual else np.zeros(n),
                theta=rng.uniform(0, 6.28, n) if dual else np.zeros(n), RE=np.full(n, 10e-6))
    C = km_coeffs_oracle(phys, W.WATER_25C)
    y = np.stack([rng.uniform(0.2, 5.0, n), rng.uniform(-20.0, 20.0, n)])
    tau = rng.uniform(0.0, 1.1, n)
    tau[:200] = np.repeat(np.arange(0, 1.25, 0.25), 40)[:200]        # exact quarter periods
    g = _eval(ens.ENS_SYS_KELLER_MIKSIS, C, tau, y)
    o = oracle.rhs(oracle.KM, C, tau, y)
    assert np.array_equal(g[0], o[0])
    y1, y2 = y
    D = np.abs(y1 - C[9] * y1 * y2 + C[4] * C[9])
    scale = (np.abs(C[0] * y1 ** -C[10]) * (1 + np.abs(C[1] * y2 / C[0])) + np.abs(C[2]) * (1 + np.abs(C[9] * y2))
             + np.abs(C[3] / y1) + np.abs(C[4] * y2 / y1) + 1.5 * y2 ** 2 * (1 + np.abs(C[9] * y2))
             + (np.abs(C[5]) + np.abs(C[6])) * (1 + np.abs(C[9] * y2)) + y1 * (np.abs(C[7]) + np.abs(C[8]))) / D
    # the oracle rounds the angle 2 pi C11 tau + C12 before its sin / cos
    ang = 2 * np.pi * (1 + np.abs(C[11])) * np.abs(tau) + np.abs(C[12])
    arg = 4 * EPS * ang * ((np.abs(C[5]) + np.abs(C[6])) * (1 + np.abs(C[9] * y2)) + y1 * (np.abs(C[7]) + np.abs(C[8]))) / D
    err = np.abs(g[1] - o[1]) / (scale + arg / (64 * EPS))
    assert err.max() < 64 * EPS, err.max()


def test_relief_valve_and_lorenz_rhs():
    rng = np.random.default_rng(5)
    n = 10000
    P = np.stack([rng.uniform(0.2, 10, n), np.full(n, 1.25), np.full(n, 10.0), np.full(n, 20.0), np.full(n, 0.8)])
    y = np.stack([rng.uniform(-0.1, 10, n), rng.uniform(-5, 5, n), rng.uniform(0, 30, n)])
    t = np.zeros(n)
    g = _eval(ens.ENS_SYS_RELIEF_VALVE, P, t, y)
    o = oracle.rhs(oracle.PRV, P, t, y)
    sc = np.abs(y).sum(0) * 30 + P[0] * 20
    assert (np.abs(g - o).max(0) / sc).max() < 8 * EPS
    L = np.stack([rng.uniform(0, 30, n), np.full(n, 10.0), np.full(n, 8 / 3)])
    y = rng.normal(scale=10, size=(3, n))
    g = _eval(ens.ENS_SYS_LORENZ, L, t, y)
    o = oracle.rhs(oracle.LORENZ, L, t, y)
    sc = (np.abs(y).max(0) + 1) ** 2 * 40
    assert (np.abs(g - o).max(0) / sc).max() < 8 * EPS
