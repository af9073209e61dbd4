"""Seeded, synthetic inputs for the ensemble workloads of arXiv 2011.01740.

This module only generates inputs (parameter grids, initial conditions,
solver settings, deterministic subsamples).  It holds none of the method's
arithmetic: Keller-Miksis coefficients, right-hand sides and steppers live in
the CUDA library (and, independently, in the CPU oracle used by the tests).
Both sides draw their inputs from here.

Workloads (the paper runs each as a sweep of one control parameter; the
shapes below follow those sweeps):
  * ``x2p``     - introductory example x' = x^2 - p, p = linspace(0.1, 1, N),
                  x0 = -0.5, dt = 0.01, 1000 RK4 steps (Sec. 3).
  * ``lorenz``  - Lorenz with sigma = 10, b = 8/3, rho = linspace(0, 21, N),
                  x = y = z = 10 at t = 0, dt = 0.01, 1000 RK4 steps (Sec. 4.1).
  * ``km``      - Keller-Miksis bubble in water at 25 C, R_E = 10 um,
                  single-frequency driving, p_A linear in [0, 2 bar] times f
                  logarithmic in [20 kHz, 1 MHz], f varying fastest; y = (1, 0)
                  at tau = 0; Cash-Karp at tol 1e-10; 64 forcing periods, max /
                  min radius per period (Sec. 4.2).
  * ``km_frequency_response`` - the paper's own Keller-Miksis run: P_A1 =
                  1.5 bar, P_A2 = 0, 46,080 values of f1 logarithmic in
                  [20 kHz, 1 MHz], 1024 transient + 64 recorded periods
                  (Sec. 4.2.1).
  * ``km_dual`` - the ``km`` sweep with a second driving component,
                  P_A2 = P_A1 / 2 at f2 = 2 f1.
  * ``prv``     - pressure relief valve, kappa = 1.25, delta = 10, beta = 20,
                  r = 0.8, q = linspace(0.2, 10, N), y = (0.2, 0, 0), t in
                  [0, 1024], tol 1e-10, event tolerance 1e-6 (Sec. 4.3).
  * ``screen``  - log-uniform p_A x f grid for surrogate screening.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED = 20201103

# Liquid and gas constants (SI).  WATER_25C is the parameter set of the
# 131,044-system sweep; WATER_PAPER repeats the constants printed in Sec. 4.2
# (viscosity read as 8.902e-4 Pa s).
WATER_25C = dict(rho=997.0, c=1497.0, mu=8.9e-4, sigma=0.0725, pv=3166.8, pinf=1.0e5, gamma=1.4)
WATER_PAPER = dict(rho=997.1, c=1497.3, mu=8.902e-4, sigma=0.072, pv=3166.8, pinf=1.0e5, gamma=1.4)

PRV_CONST = dict(kappa=1.25, delta=10.0, beta=20.0, r=0.8)


def linspace(a: float, b: float, n: int) -> np.ndarray:
    """Inclusive equidistant grid a + i (b - a) / (n - 1)."""
    if n == 1:
        return np.array([a], dtype=np.float64)
    return a + (b - a) * (np.arange(n, dtype=np.float64) / (n - 1))


def logspace(a: float, b: float, n: int) -> np.ndarray:
    """Inclusive logarithmic grid a (b / a)^(j / (n - 1))."""
    if n == 1:
        return np.array([a], dtype=np.float64)
    return a * (b / a) ** (np.arange(n, dtype=np.float64) / (n - 1))


@dataclasses.dataclass
class Tolerances:
    rtol: float = 1e-10
    atol: float = 1e-10
    dt0: float = 1e-2
    dt_min: float = 1e-14
    dt_max: float = 1e-1
    event_tol: float = 1e-6
    max_steps: int = 2_000_000_000
    n_phases: int = 0
    phase_len: float = 1.0
    t0: float = 0.0
    t1: float = 1.0
    acc_t_start: float = 0.0


# ---------------------------------------------------------------------------

def x2p(n: int = 1 << 20):
    """Sec. 3 example: params (1, n), y0 (1, n), dt, nsteps."""
    p = linspace(0.1, 1.0, n)[None, :]
    y0 = np.full((1, n), -0.5)
    return dict(params=p, y0=y0, t0=0.0, dt=0.01, nsteps=1000)


def lorenz(n: int = 16384, rho_max: float = 21.0):
    """Sec. 4.1 sweep: params (3, n) = (rho, sigma, b), y0 (3, n)."""
    rho = linspace(0.0, rho_max, n)
    params = np.stack([rho, np.full(n, 10.0), np.full(n, 8.0 / 3.0)])
    y0 = np.full((3, n), 10.0)
    return dict(params=params, y0=y0, t0=0.0, dt=0.01, nsteps=1000)


def km(m_pa: int = 362, m_f: int = 362, n_phases: int = 64, pa_max: float = 2.0e5,
       f_min: float = 2.0e4, f_max: float = 1.0e6, RE: float = 10e-6, tol: float = 1e-10,
       liquid: dict | None = None):
    """Keller-Miksis p_A x f sweep; system index = i_pA * m_f + j_f.

    Returns the physical parameters (SI) of every system; the 13 coefficients
    C0..C12 are derived from them by the solver library (or the oracle).
    """
    pa = linspace(0.0, pa_max, m_pa)
    f = logspace(f_min, f_max, m_f)
    PA, F = np.meshgrid(pa, f, indexing="ij")
    n = m_pa * m_f
    phys = dict(pA1=PA.ravel().copy(), f1=F.ravel().copy(), pA2=np.zeros(n), f2=np.zeros(n),
                theta=np.zeros(n), RE=np.full(n, RE))
    y0 = np.stack([np.ones(n), np.zeros(n)])
    tols = Tolerances(rtol=tol, atol=tol, dt0=1e-2, dt_min=1e-14, dt_max=1e-1,
                      n_phases=n_phases, phase_len=1.0, t0=0.0, t1=1.0)
    return dict(phys=phys, liquid=dict(liquid or WATER_25C), y0=y0, tol=tols,
                shape=(m_pa, m_f))


def km_frequency_response(n_f: int = 46080, pA1: float = 1.5e5, f_min: float = 2.0e4, f_max: float = 1.0e6,
                          n_transient: int = 1024, n_recorded: int = 64, RE: float = 10e-6, tol: float = 1e-10,
                          liquid: dict | None = None):
    """The Keller-Miksis frequency-response workload of Sec. 4.2: P_A1 =
    1.5 bar, P_A2 = 0, theta = 0, R_E = 10 um, n_f values of f1 log-spaced
    over 20 kHz - 1 MHz; n_transient phases are integrated and discarded,
    the maxima of the next n_recorded phases are kept (the paper: 1024 and
    64, curves of up to 46,080 frequencies)."""
    f = logspace(f_min, f_max, n_f)
    n = n_f
    phys = dict(pA1=np.full(n, pA1), f1=f, pA2=np.zeros(n), f2=np.zeros(n), theta=np.zeros(n),
                RE=np.full(n, RE))
    y0 = np.stack([np.ones(n), np.zeros(n)])
    tols = Tolerances(rtol=tol, atol=tol, dt0=1e-2, dt_min=1e-14, dt_max=1e-1,
                      n_phases=n_transient + n_recorded, phase_len=1.0, t0=0.0, t1=1.0)
    return dict(phys=phys, liquid=dict(liquid or WATER_25C), y0=y0, tol=tols, n_transient=n_transient)


def km_dual(m_pa: int = 362, m_f: int = 362, n_phases: int = 64, amp_ratio: float = 0.5, freq_ratio: float = 2.0,
            theta: float = 0.0, **kw):
    """The p_A x f sweep of km() with a second driving component: P_A2 =
    amp_ratio * P_A1 at f2 = freq_ratio * f1 with phase shift theta (the
    dual-frequency form of the Keller-Miksis forcing, Sec. 4.2)."""
    w = km(m_pa, m_f, n_phases=n_phases, **kw)
    ph = w["phys"]
    ph["pA2"] = amp_ratio * ph["pA1"]
    ph["f2"] = freq_ratio * ph["f1"]
    ph["theta"] = np.full(ph["pA1"].size, theta)
    return w


def prv(n: int = 262144, q_min: float = 0.2, q_max: float = 10.0, t1: float = 1024.0,
        tol: float = 1e-10):
    """Pressure-relief-valve q sweep: params (5, n) = (q, kappa, delta, beta, r)."""
    q = linspace(q_min, q_max, n)
    c = PRV_CONST
    params = np.stack([q, np.full(n, c["kappa"]), np.full(n, c["delta"]), np.full(n, c["beta"]),
                       np.full(n, c["r"])])
    y0 = np.stack([np.full(n, 0.2), np.zeros(n), np.zeros(n)])
    tols = Tolerances(rtol=tol, atol=tol, dt0=1e-3, dt_min=1e-14, dt_max=1.0, event_tol=1e-6,
                      t0=0.0, t1=t1, acc_t_start=t1 / 2)
    return dict(params=params, y0=y0, tol=tols)


def screen_grid(m: int = 4096, pa_min: float = 2.0e5 / 361, pa_max: float = 2.0e5,
                f_min: float = 2.0e4, f_max: float = 1.0e6):
    """Log-uniform p_A x f grid (f fastest): returns (pA, f) flattened."""
    pa = logspace(pa_min, pa_max, m)
    f = logspace(f_min, f_max, m)
    PA, F = np.meshgrid(pa, f, indexing="ij")
    return PA.ravel().copy(), F.ravel().copy()


def screen_subgrid(m: int, stride: int) -> np.ndarray:
    """Flat indices of the points of the m x m screening grid on every
    stride-th row and column (a uniform 1/stride^2 sample of the grid)."""
    r = np.arange(0, m, stride)
    return (r[:, None] * m + r[None, :]).ravel()


def screen_calibration_points(m: int, k: int, stride: int, seed: int = SEED + 3) -> np.ndarray:
    """k distinct random flat indices of the m x m screening grid that avoid
    the stride sub-grid of screen_subgrid (so a calibration sample drawn here
    never overlaps the validation sample drawn there); sorted."""
    rng = np.random.default_rng(seed)
    out = np.empty(0, dtype=np.int64)
    while out.size < k:
        cand = rng.integers(0, m * m, 2 * k)
        r, c = cand // m, cand % m
        cand = cand[(r % stride != 0) | (c % stride != 0)]
        out = np.unique(np.concatenate([out, cand]))
    return np.sort(rng.choice(out, k, replace=False))


def subsample(n: int, k: int, seed: int = SEED, strata: int = 64) -> np.ndarray:
    """Sorted stratified sample of k indices out of range(n): the index range
    is cut into `strata` equal blocks and k / strata indices are drawn from
    each without replacement."""
    if k >= n:
        return np.arange(n)
    rng = np.random.default_rng(seed)
    strata = max(1, min(strata, k))
    edges = np.linspace(0, n, strata + 1).astype(np.int64)
    per = np.full(strata, k // strata)
    per[: k - per.sum()] += 1
    out = []
    for s in range(strata):
        lo, hi = edges[s], edges[s + 1]
        take = min(per[s], hi - lo)
        out.append(lo + rng.choice(hi - lo, take, replace=False))
    return np.sort(np.concatenate(out))


def shard_rows(m_rows: int, m_cols: int, world: int, rank: int) -> np.ndarray:
    """Global system indices of rank `rank`'s shard of an m_rows x m_cols grid
    (row-major, columns fastest): every world-th row, starting at row `rank`.
    The systems are independent, so shards need no exchange while solving;
    interleaved rows give every rank the same mix of driving amplitudes, hence
    about the same cost.  The shards of ranks 0..world-1 partition the grid."""
    rows = np.arange(rank, m_rows, world)
    return (rows[:, None] * m_cols + np.arange(m_cols)[None, :]).ravel()


def take(d: dict, idx: np.ndarray) -> dict:
    """Restrict a workload's per-system arrays to the systems `idx`."""
    out = dict(d)
    for key in ("params", "y0"):
        if key in d:
            out[key] = np.ascontiguousarray(d[key][:, idx])
    if "phys" in d:
        out["phys"] = {k: np.ascontiguousarray(v[idx]) for k, v in d["phys"].items()}
    return out


# ---------------------------------------------------------------------------
# surrogate network inputs
# ---------------------------------------------------------------------------

MLP_PARAMS = 50178          # floats per ensemble member (layout: include/ens.h)
MLP_FAN_IN = [(256, 2), (128, 0), (16384, 128), (128, 0), (16384, 128), (128, 0), (16384, 128), (128, 0),
              (256, 128), (2, 0)]  # (block size, fan-in; 0 = bias) in parameter order


def mlp_params(members: int = 4, seed: int = SEED, bias_scale: float = 0.1) -> np.ndarray:
    """Seeded parameter vectors [members][50178]: weights N(0, 1/fan_in),
    biases N(0, bias_scale^2).  Member k draws from seed + k."""
    out = np.empty((members, MLP_PARAMS), dtype=np.float32)
    for k in range(members):
        rng = np.random.default_rng(seed + k)
        parts = []
        for size, fan in MLP_FAN_IN:
            scale = (1.0 / np.sqrt(fan)) if fan else bias_scale
            parts.append(rng.normal(0.0, scale, size))
        out[k] = np.concatenate(parts).astype(np.float32)
    return out


def mlp_batch(n: int, seed: int = SEED + 100):
    """Seeded inputs x in [-1, 1]^2 and targets (a smooth function, a 0/1 label)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, size=(n, 2)).astype(np.float32)
    y0 = np.sin(2.0 * x[:, 0]) * x[:, 1] + 0.3 * x[:, 0]
    y1 = (x[:, 0] + 0.5 * x[:, 1] > 0.1).astype(np.float32)
    return x, np.stack([y0, y1], axis=1).astype(np.float32)


KM_FEATURE_RANGE = (2.0e5 / 361, 2.0e5, 2.0e4, 1.0e6)   # (pA_lo, pA_hi, f_lo, f_hi)
