"""Surrogate-screened Keller-Miksis scan, assembled from C-ABI calls.

Every numerical step runs in libens.so kernels; this module only sequences
the calls and holds device buffers (torch CUDA tensors):

  1. training set: FP64 Cash-Karp solve of a p_A x f grid (ens_create /
     ens_solve), targets from the per-period maxima of the recorded periods
     (ens_km_labels), features (log p_A, log f) scaled to [-1, 1]
     (ens_km_features);
  2. an ensemble of MLPs trained on it (ens_mlp_train, BF16 tensor cores);
  3. a dense screening grid through the fused ensemble forward
     (ens_mlp_screen): mean and spread of the predicted log max radius;
  4. points whose ensemble spread exceeds `threshold` are compacted
     (ens_select_above), their coefficients planned on the device
     (ens_gather_f64, ens_km_coefficients) and re-solved in FP64; the solver's
     values replace the surrogate's there (ens_km_labels, ens_scatter_labels).
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as W


def _t(a, dev, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return t if dtype is None else t.to(dtype)


def km_solve_labels(ens, phys: dict, liquid: dict, n_phases: int, first_phase: int, dev, stream,
                    tol: float = 1e-10, spread_tol: float = 1e-4, launch=None):
    """FP64 solve of the systems `phys` (device tensors) and their labels
    y[n][2] = (ln max radius over phases >= first_phase, period-1 flag)."""
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
        ens.ens_set_launch(ctx, launch or ens.make_launch(block=128, blocks_per_sm=2, cost_order=1))
        ens.ens_solve(ctx, stream)
        st = ens.ens_sync(ctx)
        acc = torch.empty((2 * n_phases, n), dtype=torch.float64, device=dev)
        ens.ens_read(ctx, ens.ENS_ACC, acc)
        steps = int(ens.ens_read(ctx, ens.ENS_NSTEPS).sum())
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


def run(ens, train_shape=(362, 362), screen_m=1024, n_phases=64, first_phase=32, threshold=0.05,
        members=4, epochs=150, batch=1024, lr=2e-3, lr_final=2e-5, seed=W.SEED, stream=None, validate=2048,
        liquid=None, train=None):
    """Train on a train_shape grid, screen a screen_m x screen_m log grid,
    re-solve the uncertain points; returns timings, counts and errors.
    `train` = (x, y, solve_seconds, steps) reuses an existing training set."""
    import torch
    dev = torch.device("cuda")
    stream = stream or torch.cuda.Stream()
    liquid = liquid or W.WATER_25C
    out = {}
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
    # 2. training
    m = ens.ens_mlp_create(members, seed)
    try:
        t0 = time.perf_counter()
        hist = ens.ens_mlp_train(m, x_tr.shape[0], x_tr, y_tr,
                                 ens.make_train_cfg(epochs=epochs, batch=batch, lr=lr, seed=seed,
                                                    lr_final=lr_final), members,
                                 stream=stream)
        out["train_s"] = time.perf_counter() - t0
        out["train_loss_first_last"] = [float(hist[0].mean()), float(hist[-1].mean())]
        # 3. screening
        pa, f = W.screen_grid(screen_m)
        n = pa.size
        pa_d, f_d = _t(pa, dev), _t(f, dev)
        x = torch.empty((n, 2), dtype=torch.float32, device=dev)
        mean, sd, p1 = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens.ens_km_features(n, pa_d, f_d, W.KM_FEATURE_RANGE, x, stream=stream)
        ens.ens_mlp_screen(m, n, x, mean, sd, p1, stream=stream)
        stream.synchronize()
        out["screen_s"] = time.perf_counter() - t0
    finally:
        ens.ens_mlp_destroy(m)
    out["screen_points"] = n
    # 4. fallback: re-solve the uncertain points in FP64
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    t0 = time.perf_counter()
    k = ens.ens_select_above(n, sd, threshold, idx, stream=stream)
    final = mean.clone()
    fb_steps = 0
    if k > 0:
        sub = {}
        for key, src in (("pA1", pa_d), ("f1", f_d)):
            dst = torch.empty(k, dtype=torch.float64, device=dev)
            ens.ens_gather_f64(k, idx, src, dst, stream=stream)
            sub[key] = dst
        sub["pA2"] = torch.zeros(k, dtype=torch.float64, device=dev)
        sub["f2"] = torch.zeros(k, dtype=torch.float64, device=dev)
        sub["theta"] = torch.zeros(k, dtype=torch.float64, device=dev)
        sub["RE"] = torch.full((k,), 10e-6, dtype=torch.float64, device=dev)
        y_fb, st, fb_steps = km_solve_labels(ens, sub, liquid, n_phases, first_phase, dev, stream)
        ens.ens_scatter_labels(k, idx, y_fb, final, stream=stream)
        stream.synchronize()
    out["fallback_s"] = time.perf_counter() - t0
    out["fallback_points"] = int(k)
    out["fallback_fraction"] = k / n
    out["fallback_steps"] = fb_steps
    out["screened_total_s"] = out["screen_s"] + out["fallback_s"]
    # 5. error of the merged map on a validation sample solved in FP64
    if validate:
        vi = W.subsample(n, validate, seed=seed + 7)
        vphys = {"pA1": _t(pa[vi], dev), "f1": _t(f[vi], dev)}
        for key in ("pA2", "f2", "theta"):
            vphys[key] = torch.zeros(vi.size, dtype=torch.float64, device=dev)
        vphys["RE"] = torch.full((vi.size,), 10e-6, dtype=torch.float64, device=dev)
        t0 = time.perf_counter()
        y_v, st, v_steps = km_solve_labels(ens, vphys, liquid, n_phases, first_phase, dev, stream)
        v_s = time.perf_counter() - t0
        truth = y_v[:, 0].cpu().numpy().astype(np.float64)
        pred = final.cpu().numpy()[vi].astype(np.float64)
        flagged = sd.cpu().numpy()[vi] > threshold
        err = np.abs(pred - truth)
        out["validation"] = {
            "points": int(vi.size), "flagged": int(flagged.sum()),
            "abs_err_log_ratio_median": float(np.median(err)),
            "abs_err_log_ratio_p90": float(np.percentile(err, 90)),
            "abs_err_log_ratio_p99": float(np.percentile(err, 99)),
            "abs_err_unflagged_p90": float(np.percentile(err[~flagged], 90)) if (~flagged).any() else None,
            "fp64_s_per_system": v_s / vi.size,
        }
        # what a plain FP64 solve of the whole screening grid would cost: the
        # validation sample's mean steps per system at the step rate of the
        # fully occupied training solve
        rate = out["train_steps"] / out["train_solve_s"]
        out["fp64_full_grid_estimate_s"] = (v_steps / vi.size) * n / rate
        out["speedup_vs_fp64_estimate"] = out["fp64_full_grid_estimate_s"] / out["screened_total_s"]
    return out
