"""Surrogate-screened Keller-Miksis scan, assembled from C-ABI calls.

Every numerical step runs in libens.so kernels; this module sequences the
calls, holds device buffers (torch CUDA tensors) and picks one threshold:

  1. training set: FP64 Cash-Karp solve of a p_A x f grid (ens_create /
     ens_solve), targets from the per-period maxima of the recorded periods
     (ens_km_labels), features (log p_A, log f) scaled to [-1, 1]
     (ens_km_features);
  2. an ensemble of MLPs trained on it (ens_mlp_train, BF16 tensor cores);
  3. calibration of the fallback gate on a held-out sample of the screening
     grid solved in FP64: a point goes back to the solver when the ensemble
     spread exceeds `threshold` (the configured spread gate), or when the
     predicted map is steep there (ens_feature_stencil, ens_mlp_screen,
     ens_stencil_gradient).  The steepness threshold is the largest for which
     the sample's unflagged |error| stays within `bound` at the `quantile`;
  4. the dense screening grid through the fused ensemble forward
     (ens_mlp_screen) and its steepness (ens_grid_gradient);
  5. the points either gate flags are compacted (ens_select_gate), their
     coefficients planned on the device (ens_gather_f64, ens_km_coefficients)
     and re-solved in FP64; the solver's values replace the surrogate's there
     (ens_km_labels, ens_scatter_labels);
  6. validation on a uniform sub-grid of the screening grid solved in FP64
     (disjoint from the calibration sample): the error of the merged map,
     the period-1 output against the solver's label, and the measured FP64
     time of that sub-grid, which scales to the whole grid.
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as W


def _t(a, dev, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return t if dtype is None else t.to(dtype)


def _phys(pa, f, dev):
    import torch
    n = pa.numel()
    ph = {"pA1": pa, "f1": f}
    for key in ("pA2", "f2", "theta"):
        ph[key] = torch.zeros(n, dtype=torch.float64, device=dev)
    ph["RE"] = torch.full((n,), 10e-6, dtype=torch.float64, device=dev)
    return ph


def km_solve_labels(ens, phys: dict, liquid: dict, n_phases: int, first_phase: int, dev, stream,
                    tol: float = 1e-10, spread_tol: float = 1e-4, launch=None, per_system=None):
    """FP64 solve of the systems `phys` (device tensors) and their labels
    y[n][2] = (ln max radius over phases >= first_phase, period-1 flag).
    per_system (a list) receives the accepted steps of every system."""
    import torch
    n = phys["pA1"].numel()
    C = ens.ens_km_coefficients(phys["pA1"], phys["f1"], phys["pA2"], phys["f2"], phys["theta"], phys["RE"],
                                liquid, stream=stream)
    y0 = torch.zeros((2, n), dtype=torch.float64, device=dev)
    y0[0] = 1.0
    stream.synchronize()
    ttol = ens.make_tol(rtol=tol, atol=tol, dt0=1e-2, dt_min=1e-14, dt_max=1e-1, n_phases=n_phases,
                        timeout_s=1800.0)
    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, n, C, y0, (0.0, 1.0), ens.ENS_RKCK45, ttol)
    try:
        ens.ens_set_launch(ctx, launch or ens.make_launch(block=160, blocks_per_sm=1, cost_order=1))
        ens.ens_solve(ctx, stream)
        st = ens.ens_sync(ctx)
        acc = torch.empty((2 * n_phases, n), dtype=torch.float64, device=dev)
        ens.ens_read(ctx, ens.ENS_ACC, acc)
        nacc = ens.ens_read(ctx, ens.ENS_NSTEPS)
        steps = int(nacc.sum())
        if per_system is not None:
            per_system.append(nacc)
    finally:
        ens.ens_destroy(ctx)
    y = torch.empty((n, 2), dtype=torch.float32, device=dev)
    ens.ens_km_labels(n, acc, n_phases, first_phase, spread_tol, y, stream=stream)
    stream.synchronize()
    return y, st, steps


def training_set_from_acc(ens, km: dict, acc, n_phases: int, first_phase: int, dev, stream,
                          spread_tol: float = 1e-4):
    """Features and labels of an already solved p_A x f grid (acc: device
    accessories [2 n_phases][n]); the p_A = 0 row is left out."""
    import torch
    keep = np.nonzero(km["phys"]["pA1"] > 0)[0]
    n = km["phys"]["pA1"].size
    y_all = torch.empty((n, 2), dtype=torch.float32, device=dev)
    ens.ens_km_labels(n, acc, n_phases, first_phase, spread_tol, y_all, stream=stream)
    pa = _t(km["phys"]["pA1"][keep], dev)
    f = _t(km["phys"]["f1"][keep], dev)
    x = torch.empty((keep.size, 2), dtype=torch.float32, device=dev)
    ens.ens_km_features(keep.size, pa, f, W.KM_FEATURE_RANGE, x, stream=stream)
    stream.synchronize()
    return x, y_all[_t(keep, dev)].contiguous()


def calibrate_gradient_gate(err: np.ndarray, sd: np.ndarray, g: np.ndarray, spread_thr: float, bound: float,
                            quantile: float = 99.0, min_kept: int = 200) -> float:
    """The largest steepness threshold t for which the calibration points
    passing both gates (spread <= spread_thr and steepness <= t) have their
    |error| `quantile` within `bound`; 0 when none does (then every point
    with a nonzero slope goes to the solver)."""
    ok = sd <= spread_thr
    cand = np.unique(np.quantile(g[ok], np.linspace(0.0, 1.0, 801))) if ok.any() else np.empty(0)
    for t in cand[::-1]:
        kept = ok & (g <= t)
        if kept.sum() < min_kept:
            break
        if np.percentile(err[kept], quantile) <= bound:
            return float(t)
    return 0.0


def run(ens, train_shape=(362, 362), screen_m=1024, n_phases=64, first_phase=32, threshold=0.05,
        bound=0.05, quantile=99.0, calib_points=16384, val_stride=4, slope_spacing=2.0 / 1023, members=4,
        epochs=2400, batch=8192, lr=6e-3, lr_final=2e-5, seed=W.SEED, stream=None, liquid=None, train=None,
        fallback_launch=None):
    """Train on a train_shape grid, calibrate the fallback gate, screen a
    screen_m x screen_m log grid, re-solve the flagged points, validate on the
    every-val_stride-th sub-grid; returns timings, counts and errors.  The
    steepness is taken over about `slope_spacing` in feature units (a whole
    number of grid steps; by default the step of a 1024-point axis): over a
    finer spacing the rounding noise of the network's output, not its slope,
    sets the difference.  `train` = (x, y, solve_seconds, steps) reuses an
    existing training set."""
    import torch
    dev = torch.device("cuda")
    stream = stream or torch.cuda.Stream()
    liquid = liquid or W.WATER_25C
    out = {"spread_threshold": threshold, "bound": {"quantile": quantile, "abs_err_log_ratio": bound}}
    # 1. training data (the p_A = 0 row has no logarithm and is left out)
    if train is not None:
        x_tr, y_tr, out["train_solve_s"], out["train_steps"] = train
        out["train_systems"] = int(x_tr.shape[0])
    else:
        km = W.km(train_shape[0], train_shape[1], n_phases=n_phases, liquid=liquid)
        keep = km["phys"]["pA1"] > 0
        phys = {k: _t(v[keep], dev) for k, v in km["phys"].items()}
        t0 = time.perf_counter()
        y_tr, st, steps = km_solve_labels(ens, phys, liquid, n_phases, first_phase, dev, stream)
        out["train_solve_s"] = time.perf_counter() - t0
        out["train_systems"] = int(keep.sum())
        out["train_steps"] = steps
        x_tr = torch.empty((int(keep.sum()), 2), dtype=torch.float32, device=dev)
        ens.ens_km_features(x_tr.shape[0], phys["pA1"], phys["f1"], W.KM_FEATURE_RANGE, x_tr, stream=stream)
        stream.synchronize()
    pa, f = W.screen_grid(screen_m)
    n = pa.size
    d = 2.0 / (screen_m - 1)                 # grid spacing in feature units (both axes span [-1, 1])
    gstride = max(1, int(round(slope_spacing / d)))
    ds = gstride * d                         # the distance the steepness is taken over
    out["slope_spacing"] = ds
    m = ens.ens_mlp_create(members, seed)
    try:
        # 2. training
        t0 = time.perf_counter()
        hist = ens.ens_mlp_train(m, x_tr.shape[0], x_tr, y_tr,
                                 ens.make_train_cfg(epochs=epochs, batch=batch, lr=lr, seed=seed,
                                                    lr_final=lr_final), members, stream=stream)
        out["train_s"] = time.perf_counter() - t0
        out["train_loss_first_last"] = [float(hist[0].mean()), float(hist[-1].mean())]
        # 3. calibration of the steepness gate on held-out solved points
        t0 = time.perf_counter()
        ci = W.screen_calibration_points(screen_m, calib_points, val_stride, seed=seed + 3)
        kc = ci.size
        cpa, cf = _t(pa[ci], dev), _t(f[ci], dev)
        y_c, _, _ = km_solve_labels(ens, _phys(cpa, cf, dev), liquid, n_phases, first_phase, dev, stream,
                                    launch=fallback_launch)
        xc = torch.empty((kc, 2), dtype=torch.float32, device=dev)
        ens.ens_km_features(kc, cpa, cf, W.KM_FEATURE_RANGE, xc, stream=stream)
        xs = torch.empty((5 * kc, 2), dtype=torch.float32, device=dev)
        ens.ens_feature_stencil(kc, xc, ds, ds, xs, stream=stream)
        mu5, sd5, p15 = [torch.empty(5 * kc, dtype=torch.float32, device=dev) for _ in range(3)]
        ens.ens_mlp_screen(m, 5 * kc, xs, mu5, sd5, p15, stream=stream)
        gc = torch.empty(kc, dtype=torch.float32, device=dev)
        ens.ens_stencil_gradient(kc, mu5, ds, ds, gc, stream=stream)
        stream.synchronize()
        err_c = np.abs(mu5[:kc].cpu().numpy().astype(np.float64) - y_c[:, 0].cpu().numpy())
        sd_c, g_c = sd5[:kc].cpu().numpy(), gc.cpu().numpy()
        g_thr = calibrate_gradient_gate(err_c, sd_c, g_c, threshold, bound, quantile)
        kept_c = (sd_c <= threshold) & (g_c <= g_thr)
        out["calibration"] = {"points": int(kc), "solve_and_fit_s": time.perf_counter() - t0,
                              "gradient_threshold": g_thr, "kept_fraction": float(kept_c.mean()),
                              "unflagged_err_quantile": float(np.percentile(err_c[kept_c], quantile))
                              if kept_c.any() else None,
                              "spread_only_err_p99": float(np.percentile(err_c[sd_c <= threshold], 99))
                              if (sd_c <= threshold).any() else None,
                              "corr_err_spread": float(np.corrcoef(err_c, sd_c)[0, 1]),
                              "corr_err_gradient": float(np.corrcoef(err_c, g_c)[0, 1])}
        # 4. screening and steepness of the predicted map
        pa_d, f_d = _t(pa, dev), _t(f, dev)
        x = torch.empty((n, 2), dtype=torch.float32, device=dev)
        mean, sd, p1, g = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(4)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens.ens_km_features(n, pa_d, f_d, W.KM_FEATURE_RANGE, x, stream=stream)
        ens.ens_mlp_screen(m, n, x, mean, sd, p1, stream=stream)
        ens.ens_grid_gradient(screen_m, screen_m, gstride, mean, d, d, g, stream=stream)
        stream.synchronize()
        out["screen_s"] = time.perf_counter() - t0
    finally:
        ens.ens_mlp_destroy(m)
    out["screen_points"] = n
    # 5. fallback: re-solve the flagged points in FP64
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    t0 = time.perf_counter()
    k = ens.ens_select_gate(n, sd, threshold, g, g_thr, idx, stream=stream)
    final = mean.clone()
    fb_steps = 0
    if k > 0:
        sub = {}
        for key, src in (("pA1", pa_d), ("f1", f_d)):
            dst = torch.empty(k, dtype=torch.float64, device=dev)
            ens.ens_gather_f64(k, idx, src, dst, stream=stream)
            sub[key] = dst
        y_fb, st, fb_steps = km_solve_labels(ens, _phys(sub["pA1"], sub["f1"], dev), liquid, n_phases,
                                             first_phase, dev, stream, launch=fallback_launch)
        ens.ens_scatter_labels(k, idx, y_fb, final, stream=stream)
        stream.synchronize()
    out["fallback_s"] = time.perf_counter() - t0
    out["fallback_points"] = int(k)
    out["fallback_fraction"] = k / n
    out["fallback_by_spread"] = int((sd > threshold).sum())
    out["fallback_steps"] = fb_steps
    out["screened_total_s"] = out["screen_s"] + out["fallback_s"]
    out["fixed_s"] = out["train_solve_s"] + out["train_s"] + out["calibration"]["solve_and_fit_s"]
    # 6. validation on the uniform sub-grid, solved in FP64
    vi = W.screen_subgrid(screen_m, val_stride)
    vi_d = _t(vi, dev)
    t0 = time.perf_counter()
    v_nacc = []
    y_v, st, v_steps = km_solve_labels(ens, _phys(_t(pa[vi], dev), _t(f[vi], dev), dev), liquid, n_phases,
                                       first_phase, dev, stream, launch=fallback_launch, per_system=v_nacc)
    v_s = time.perf_counter() - t0
    truth = y_v[:, 0].cpu().numpy().astype(np.float64)
    label = y_v[:, 1].cpu().numpy() > 0.5
    pred = final[vi_d].cpu().numpy().astype(np.float64)
    flagged = np.zeros(n, dtype=bool)
    flagged[idx[:k].cpu().numpy()] = True
    fl = flagged[vi]
    err = np.abs(pred - truth)
    p1v = p1[vi_d].cpu().numpy() > 0.5
    q = lambda a, p: float(np.percentile(a, p)) if a.size else None
    out["validation"] = {
        "points": int(vi.size), "grid": [screen_m // val_stride + (screen_m % val_stride > 0)] * 2,
        "flagged": int(fl.sum()), "fp64_s": v_s, "fp64_steps": v_steps, "status": int(st),
        "err_all": {"median": q(err, 50), "p90": q(err, 90), "p99": q(err, 99), "max": float(err.max())},
        "err_unflagged": {"median": q(err[~fl], 50), "p90": q(err[~fl], 90), "p99": q(err[~fl], 99),
                          "max": float(err[~fl].max()) if (~fl).any() else None,
                          f"p{quantile:g}": q(err[~fl], quantile)},
        "err_flagged_max": float(err[fl].max()) if fl.any() else None,
        "period1_fraction": float(label.mean()),
        "period1_error_rate_unflagged": float(np.mean(p1v[~fl] != label[~fl])) if (~fl).any() else None,
    }
    # error against cost for other bounds, from the same calibration and
    # validation solves: the gate each bound would give, its unflagged error
    # on the validation sub-grid, the share of the FP64 work (steps) its
    # flagged points carry, and the speedup that share implies
    steps_v = v_nacc[0].astype(np.float64)
    sd_v, g_v = sd[vi_d].cpu().numpy(), g[vi_d].cpu().numpy()
    curve = []
    for b in (0.02, 0.03, 0.05, 0.1, 0.2):
        tb = calibrate_gradient_gate(err_c, sd_c, g_c, threshold, b, quantile)
        fb = (sd_v > threshold) | (g_v > tb)
        work = float(steps_v[fb].sum() / steps_v.sum())
        curve.append({"bound": b, "gradient_threshold": tb, "flagged": float(fb.mean()), "fp64_work_share": work,
                      f"unflagged_p{quantile:g}": q(err[~fb], quantile),
                      "speedup_est": 1.0 / (work + out["screen_s"] / (v_s * n / vi.size))})
    out["bound_curve"] = curve
    # the plain FP64 solve of the whole grid: the uniform sub-grid's measured
    # time scaled by the number of points
    out["fp64_grid_estimate_s"] = v_s * n / vi.size
    out["speedup"] = out["fp64_grid_estimate_s"] / out["screened_total_s"]
    out["speedup_incl_fixed"] = out["fp64_grid_estimate_s"] / (out["screened_total_s"] + out["fixed_s"])
    return out
