"""Benchmark of the ensemble ODE solver (arXiv 2011.01740 method) on GB300.

One step = one full solve of the Keller-Miksis ensemble: a 362 x 362 grid of
driving amplitude p_A (linear, 0-2 bar) and frequency f (logarithmic,
20 kHz - 1 MHz), 131,044 bubbles, Cash-Karp 4(5) at rtol = atol = 1e-10,
64 forcing periods with the per-period max / min radius recorded (Sec. 4.2).
The metric is accepted RK system-steps per second.  With --gpus N (torchrun)
every rank solves its own 131,044-system slice of a 362N x 362 grid (p_A rows
interleaved across ranks), so the work per GPU is fixed (weak scaling) and no
data crosses ranks during the solve.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2011_01740_gb300 import workloads as W  # noqa: E402

# FP64 flops (DFMA = 2, DADD = DMUL = 1) executed per Cash-Karp trial step of
# the Keller-Miksis kernel, and per RK4 step of the x' = x^2 - p and Lorenz
# kernels, from the ncu instruction counters of profiles/ (None until
# measured: the roofline then reports achieved = null).
FLOPS_PER_KM_TRIAL = 340.19  # 135.68 DFMA + 65.86 DMUL + 2.98 DADD per trial (profiles/)
# all FP64 thread instructions per trial, for the FP64 pipe's issue fraction
FP64_INST_PER_KM_TRIAL = 204.52
# The same trial in its all-FP64 form (the forcing's sine and cosine, the
# fifth root, the polytropic power and the error norm's reciprocals as FP64
# arithmetic: 232.61 DFMA + 121.70 DMUL + 2.98 DADD, profiles/); the
# fixed-point evaluations on the integer pipe take 250 of these flops off the
# FP64 pipe.  Reported beside the executed count as the trial's FP64-form work.
FLOPS_FP64_FORM_KM_TRIAL = 589.91
# DRAM bytes (read + write) of one benchmarked Keller-Miksis launch, from the
# one-pass ncu capture in profiles/ (inputs 15.7 MB read once, 134 MB of
# per-period accessories written once); None once the kernel changes.
KM_LAUNCH_DRAM_BYTES = 40354816 + 120015104
FLOPS_PER_X2P_STEP = 21.0     # 10 DFMA + 1 DADD (Sec. 3.2.2 counters; kernel counted by ncu)
FLOPS_PER_LORENZ_STEP = 75.0  # 30 DFMA + 8 DMUL + 7 DADD per step of the fast kernel
# executed flops per trial of the other adaptive kernels (ncu counts,
# profiles/; None until measured: their fractions are then null)
FLOPS_PER_VALVE_TRIAL = 219.10        # FP64: 84.83 DFMA + 35.34 DMUL + 14.10 DADD, ck_events_kernel
# the valve trial in its all-FP64 form (square root, fifth root and reciprocals
# as FP64 arithmetic: 115.0 DFMA + 57.5 DMUL + 14.1 DADD, profiles/)
FLOPS_FP64_FORM_VALVE_TRIAL = 301.59
FLOPS_FP32_PER_FP32C_TRIAL = 1516.0   # FP32: 441.1 FFMA + 162.4 FMUL + 471.4 FADD, ck_phased_fp32c_kernel
FLOPS_FP32_PER_DF_TRIAL = 5277.6      # FP32: 746.1 FFMA + 454.9 FMUL + 3330.5 FADD, ck_phased_df_kernel
FLOPS_FP32_PER_DF_VALVE_TRIAL = 3173.5  # FP32, ck_events_df_kernel
# FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
FP32_PEAK = 152 * 128 * 2.0 * 2070.0e6

# FP64 peak: 152 SMs x 4 FP64 flop/clk/SM (2 DFMA lanes) x 2.07 GHz = 1.2586
# TFLOP/s, the nominal 1.25 TFLOP/s of the part at its maximum SM clock.
SMS = 152
FP64_FLOP_PER_CLK_SM = 4.0
SM_MAX_MHZ = 2070.0
FP64_PEAK = SMS * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6
FP64_INST_PEAK = SMS * 2.0 * SM_MAX_MHZ * 1e6   # FP64 thread instructions per second

WORKLOAD = "keller_miksis_362x362_pA0-2bar_f20k-1M_log_64periods_ck45_tol1e-10_fp64"
METRIC = "accepted RK system-steps/s (Keller-Miksis 362x362 p_A x f grid, Cash-Karp 1e-10, 64 periods, FP64)"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def km_slice(world: int, rank: int, m: int = 362, n_phases: int = 64):
    """Rank `rank`'s share of a (m world) x m grid: every world-th p_A row."""
    full = W.km(m * world, m, n_phases=n_phases)
    return W.take(full, W.shard_rows(m * world, m, world, rank))


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        cmd = ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            return
        try:
            while not self._stop.is_set():
                line = p.stdout.readline()
                if not line:
                    break
                self.samples.append([x.strip() for x in line.split(",")])
        finally:
            p.terminate()
            try:
                p.wait(timeout=2)
            except Exception:
                p.kill()

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=3)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if len(s) > 4 + k and s[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        busy = [v for v in sm if v > 0]
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    import paper_2011_01740_gb300 as ens

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod

    def barrier():
        if dist is not None:
            dist.barrier()

    km = km_slice(world, rank, n_phases=args.phases)
    ph = km["phys"]
    n = ph["pA1"].size
    t = km["tol"]
    tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                       n_phases=t.n_phases, phase_len=t.phase_len, timeout_s=900.0)
    stream = torch.cuda.Stream()
    dev = torch.device("cuda", local)
    # inputs resident in HBM before timing: coefficients planned on the device
    phys_d = [torch.from_numpy(ph[k]).to(dev) for k in ("pA1", "f1", "pA2", "f2", "theta", "RE")]
    C_d = ens.ens_km_coefficients(*phys_d, km["liquid"], stream=stream)
    y0_d = torch.from_numpy(km["y0"]).to(dev)
    stream.synchronize()
    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, n, C_d, y0_d, (0.0, 1.0), ens.ENS_RKCK45, tol)
    hand = ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=args.block, blocks_per_sm=args.bps, use_graph=1,
                           cost_order=args.cost_order)
    ens.ens_set_launch(ctx, hand)
    tune = None
    if not args.no_tune:
        # the project's autotuner picks the launch on 1/8 of the horizon of every system
        t0 = time.perf_counter()
        ens.ens_autotune(ctx, stream)
        tune = {"s": time.perf_counter() - t0, "table": ens.ens_autotune_table(ctx)}
    launch = ens.ens_get_launch(ctx)
    kernels_per_solve = 1 + (4 if launch.cost_order else 0)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    for _ in range(args.warmup):
        ens.ens_solve(ctx, stream)
        if ens.ens_sync(ctx) != ens.ENS_OK:
            raise RuntimeError(ens.ens_last_error(ctx))

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    kernel_ms_steps = []
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()                       # evict L2 between timed steps
            ev[k][0].record(stream)
            ens.ens_solve(ctx, stream)
            ev[k][1].record(stream)
            # the main kernel's own events (recorded by the library on this
            # stream) are read before the next solve records them again
            stream.synchronize()
            try:
                kernel_ms_steps.append(ens.ens_kernel_ms(ctx))
            except ens.EnsError:
                kernel_ms_steps.append(None)
        stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    st = ens.ens_sync(ctx)
    if st != ens.ENS_OK:
        raise RuntimeError(f"solve status {st}: {ens.ens_last_error(ctx)}")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    nacc = ens.ens_read(ctx, ens.ENS_NSTEPS)
    nrej = ens.ens_read(ctx, ens.ENS_NREJ)
    steps_local = float(nacc.sum()) * args.steps
    trials_local = float(nacc.sum() + nrej.sum())

    # whole-job aggregate: all ranks' steps over the slowest rank's time
    if dist is not None:
        tt = torch.tensor([total_ms, steps_local], dtype=torch.float64, device=dev)
        mx = tt.clone()
        dist.all_reduce(mx[0:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(tt[1:2], op=dist.ReduceOp.SUM)
        total_ms_max, steps_all = float(mx[0]), float(tt[1])
    else:
        total_ms_max, steps_all = total_ms, steps_local
    value = steps_all / (total_ms_max / 1e3)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(ens, ctx, km, stream, args, dist, dev, world)

    # ---- roofline of the dominant kernel ----
    if all(k is not None for k in kernel_ms_steps):
        kernel_ms, kernel_src = float(np.mean(kernel_ms_steps)), "main-kernel CUDA events (ens_kernel_ms)"
    else:
        kernel_ms, kernel_src = total_ms / args.steps, "whole solve (pilot and ordering included)"
    roofline = km_roofline(trials_local, kernel_ms, steps_local / args.steps)
    roofline["duration_source"] = kernel_src

    secondary = {}
    # the tuned launch against the hand-picked one on the full solve (one
    # solve each, main-kernel time)
    if tune is not None:
        launch_hand_ms = None
        if rank == 0 and world == 1 and not args.quick:
            ens.ens_set_launch(ctx, hand)
            ens.ens_solve(ctx, stream)
            ens.ens_sync(ctx)
            launch_hand_ms = ens.ens_kernel_ms(ctx)
            ens.ens_set_launch(ctx, launch)
        secondary["headline_tuning"] = {
            "chosen": launch.as_dict(), "tuner_s": tune["s"], "tuned_kernel_ms": kernel_ms,
            "hand_launch": hand.as_dict(), "hand_kernel_ms": launch_hand_ms,
            "table": [[r["launch"]["mode"], r["launch"]["block"], r["launch"]["blocks_per_sm"],
                       r["launch"]["cost_order"], round(r["ms"], 2)] for r in tune["table"]],
            "table_columns": ["mode", "block", "blocks_per_sm", "cost_order", "ms (1/8 horizon)"]}
    # single-GPU secondaries: at N > 1 they would hold every rank's GPU while
    # rank 0 alone works
    if rank == 0 and world == 1 and not args.quick:
        secondary.update(run_secondary(ens, torch, stream, dev, tuned=not args.no_tune))
        secondary["km_1024x1024_precisions"] = run_config4(ens, torch, stream, dev, tuned=not args.no_tune)
        secondary["km_work_precision_16384f"] = run_work_precision(ens, torch, stream, dev)
        secondary["km_frequency_response_46080f"] = run_frequency_response(ens, torch, stream, dev)
        secondary["km_dual_frequency_362x362"] = run_dual_frequency(ens, torch, stream, dev, launch)
        secondary["km_lyapunov_362x362"] = run_lyapunov(ens, torch, stream, dev, C_d, km, launch)
        secondary["km_dopri5_362x362"] = run_dopri5(ens, torch, stream, dev, ctx, C_d, y0_d, km, tol, launch,
                                                    total_ms / args.steps)
        secondary["km_fp32x2_362x362"] = run_fp32x2(ens, torch, stream, dev, ctx, C_d, y0_d, km, tol,
                                                    total_ms / args.steps)
        secondary["km_surrogate_screen"] = run_screen(ens, torch, stream, dev, ctx, km, total_ms / args.steps,
                                                      steps_local / args.steps, args)

    # the same kernel-level rate against the FP64 rate this GPU reached on the
    # x' = x^2 - p calibration kernel (10 DFMA + 1 DADD per step, Sec. 3)
    cal = secondary.get("x2p_rk4_calibration")
    if cal and roofline["achieved"]:
        roofline["calibration_tflops"] = cal["fp64_tflops"]
        roofline["frac_of_calibration"] = roofline["achieved"] / cal["fp64_tflops"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(km, args.cpu_seconds)

    ens.ens_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "system-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (deterministic parameter grid; no dataset)",
            "config": {"workload": WORKLOAD, "systems_per_gpu": n, "systems": n * world,
                       "grid": [362 * world, 362], "n_phases": args.phases,
                       "launch": launch.as_dict(), "launch_source": "ens_autotune" if tune else "hand-picked",
                       "l2": "256 MiB buffer written between timed steps (inputs 14 MB < L2)",
                       "parallelism": f"systems sharded over {world} GPU(s), no collective in the solve"},
            "accepted_steps_per_solve": steps_local / args.steps,
            "trial_steps_per_solve": trials_local,
            "step_ms": step_ms,
            "secondary": secondary,
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "gpu_launches": kernels_per_solve * args.steps,
        }
        # last key: one compact record per workload configuration, so that the
        # tail of the line carries every configuration's number
        line["configs"] = configs_summary(value, roofline, secondary, n)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def km_roofline(trials: float, kernel_ms: float, accepted: float) -> dict:
    """Roofline of the FP64 Keller-Miksis phase kernel: executed FP64 flops
    per trial (ncu counts, profiles/) x trials / main-kernel time against the
    FP64 peak derived from the clocks; with the FP64 instruction issue
    fraction and the accepted share of the trials."""
    achieved = FLOPS_PER_KM_TRIAL * trials / (kernel_ms / 1e3) / 1e12 if FLOPS_PER_KM_TRIAL else None
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK / 1e12, "unit": "TFLOP/s",
            "frac": (achieved / (FP64_PEAK / 1e12)) if achieved else None,
            "traffic": KM_LAUNCH_DRAM_BYTES, "kernel": "ck_phased_kernel<KellerMiksis<false, true>>",
            "peak_source": "derived: 152 SMs x 4 FP64 flop/clk/SM x 2070 MHz (nominal 1.25 TFLOP/s)",
            "flops_per_trial": FLOPS_PER_KM_TRIAL, "trials_per_launch": trials,
            "kernel_ms": kernel_ms,
            "fp64_inst_per_trial": FP64_INST_PER_KM_TRIAL,
            "fp64_issue_frac": (FP64_INST_PER_KM_TRIAL * trials / (kernel_ms / 1e3) / FP64_INST_PEAK
                                if FP64_INST_PER_KM_TRIAL else None),
            # the trial's flops in its all-FP64 form over the same time: what an
            # FP64-only kernel would have to reach to match this one
            "fp64_form_frac": FLOPS_FP64_FORM_KM_TRIAL * trials / (kernel_ms / 1e3) / FP64_PEAK,
            # the share of the work spent on accepted steps (rejected trials are discarded)
            "useful_frac": accepted / trials if trials else None}


def _tune_table(ens, ctx):
    """The context's last tuning: [mode, block, blocks_per_sm, cost_order,
    systems_per_thread, ms, horizon fraction] per candidate."""
    return [[r["launch"]["mode"], r["launch"]["block"], r["launch"]["blocks_per_sm"], r["launch"]["cost_order"],
             r["launch"]["systems_per_thread"], round(r["ms"], 3), r["horizon_frac"]]
            for r in ens.ens_autotune_table(ctx)]


def _r(x, digits=4):
    """Round to `digits` significant digits (None passes through)."""
    if x is None:
        return None
    if isinstance(x, (list, tuple)):
        return [_r(v, digits) for v in x]
    if isinstance(x, dict):
        return {k: _r(v, digits) for k, v in x.items()}
    if isinstance(x, (int, np.integer)) and not isinstance(x, bool):
        return int(x)
    if isinstance(x, (float, np.floating)):
        return float(f"{float(x):.{digits}g}")
    return x


def _shape(L: dict) -> str:
    """Launch shape in a few characters: warps per SM (persistent) or block x
    systems per thread (plain), 'lf' for longest-first claiming."""
    if L.get("mode") == 1:
        return f"{L['block'] // 32 * L['blocks_per_sm']}w/SM" + (" lf" if L.get("cost_order") else "")
    return f"plain b{L['block']}" + (f" spt{L['systems_per_thread']}" if L.get("systems_per_thread", 1) > 1 else "")


def configs_summary(value, roofline, sec, n_headline):
    """One compact record per workload configuration (values rounded; rates
    in accepted system-steps/s unless a unit is given; s = seconds; frac =
    fraction of the FP64 (FP32 for the fp32c / df variants) flop peak)."""
    out = {}
    lor = sec.get("lorenz_rk4_16384")
    if lor:
        out["c1_lorenz_rk4_16384"] = {
            "value": _r(lor["value"]), "frac": _r(lor["fp64_frac"], 3), "launch": _shape(lor["launch"]),
            "parity": "strict bit-exact, fma <=1e-12",
            "N_frac": {str(k): _r(v["fp64_frac"], 3) for k, v in sec.get("lorenz_rk4_n_sweep", {}).items()}}
    ht = sec.get("headline_tuning")
    out["c2_km_362sq_fp64"] = {
        "value": _r(value), "frac": _r(roofline.get("frac"), 3), "issue_frac": _r(roofline.get("fp64_issue_frac"), 3),
        "n": n_headline, "launch": _shape(ht["chosen"]) if ht else None,
        "hand_over_tuned": _r(ht["hand_kernel_ms"] / ht["tuned_kernel_ms"], 3) if ht and ht.get("hand_kernel_ms") else None,
        "parity": "acc <=1e-8"}
    v = sec.get("relief_valve_262144")
    if v:
        out["c3_valve_262144_fp64"] = {"value": _r(v["value"]), "s": _r(v["ms"] / 1e3), "frac": _r(v.get("fp64_frac"), 3),
                                       "form_frac": _r(v.get("fp64_form_frac"), 3),
                                       "launch": _shape(v["launch"]), "parity": "events exact, acc <=1e-8"}
        if v.get("fp32x2"):
            out["c3_valve_262144_fp64"]["df"] = _r({k: v["fp32x2"][k] for k in ("s", "speedup", "err_p99", "fp32_frac")},
                                                   3)
    c4 = sec.get("km_1024x1024_precisions")
    if c4:
        names = (("fp64_1e-10", "fp64_tol1e-10"), ("fp64_1e-8", "fp64_tol1e-8"), ("fp32c_1e-8", "fp32c_tol1e-8"),
                 ("df_1e-10", "fp32x2_tol1e-10"))
        out["c4_km_1024sq"] = {
            "s": {a: _r(c4[b]["ms"] / 1e3, 3) for a, b in names},
            "frac": {a: _r(c4[b].get("frac"), 3) for a, b in names if a != "fp64_1e-8"},
            "x_fp32c_same_tol": _r(c4["speedup_fp32c_vs_fp64_same_tol"], 3),
            "x_fp32c_vs_1e-10": _r(c4["speedup_fp32c_vs_fp64_1e-10"], 3),
            "x_df": _r(c4["speedup_fp32x2_vs_fp64"], 3),
            "err_fp32c": _r(c4["fp32c_vs_fp64_same_tol"], 2),
            "err_df": _r({k: c4["fp32x2_vs_fp64"][k] for k in ("median", "p99", "max")}, 2)}
    sc = sec.get("km_surrogate_screen")
    if sc:
        val = sc["validation"]
        out["c5_screen_4096sq"] = {
            "value": _r(sc["value"]), "unit": "points/s", "bound_p99": sc["bound"]["abs_err_log_ratio"],
            "err_unflagged": _r({k: val["err_unflagged"][k] for k in ("p90", "p99", "max")}, 3),
            "fallback": _r(sc["fallback_fraction"], 3), "p1_err": _r(val["period1_error_rate_unflagged"], 3),
            "x": _r(sc["speedup"], 3), "x_incl_fixed": _r(sc["speedup_incl_fixed"], 3),
            "fp64_1024sq_s": _r(val["fp64_s"], 3),
            "x_est_by_bound": {str(c["bound"]): _r(c["speedup_est"], 3) for c in sc.get("bound_curve", [])}}
    return out


def run_e2e(ens, ctx, km, stream, args, dist=None, dev=None, world=1):
    """Same metric through the public API with HOST buffers: host planner,
    host->device inputs, solve, device->host accessories and status.  Every
    rank runs its shard; a step's time is the slowest rank's (barrier on both
    sides), its steps and copied bytes are summed over ranks."""
    import torch
    ph = km["phys"]
    n = ph["pA1"].size
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in ph.items()}
    y0_h = torch.from_numpy(km["y0"]).pin_memory()
    rows = ens.ens_acc_rows(ctx)
    acc_h = torch.empty((rows, n), dtype=torch.float64).pin_memory()
    st_h = torch.empty((n,), dtype=torch.int32).pin_memory()
    C_h = torch.empty((13, n), dtype=torch.float64).pin_memory()
    times = []
    steps = 0.0
    for k in range(args.e2e_steps):
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        ens.ens_km_coefficients(*[pinned[k2] for k2 in ("pA1", "f1", "pA2", "f2", "theta", "RE")],
                                km["liquid"], out=C_h, stream=stream)
        ens.ens_set_inputs(ctx, C_h, y0_h, stream)
        ens.ens_solve(ctx, stream)
        st = ens.ens_sync(ctx)
        ens.ens_read(ctx, ens.ENS_ACC, acc_h)
        ens.ens_read(ctx, ens.ENS_STATUS, st_h)
        times.append(time.perf_counter() - t0)
        if st != ens.ENS_OK:
            raise RuntimeError(ens.ens_last_error(ctx))
        steps += float(ens.ens_read(ctx, ens.ENS_NSTEPS).sum())
    if dist is not None:
        t = torch.tensor(times + [steps], dtype=torch.float64, device=dev)
        tmax, tsum = t.clone(), t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        times = [float(v) for v in tmax[:-1]]
        steps = float(tsum[-1])
    return {"value": steps / sum(times), "unit": "system-steps/s",
            "h2d_bytes_per_step": int((13 + 2) * n * 8) * world,
            "d2h_bytes_per_step": int(rows * n * 8 + n * 4) * world,
            "steps": args.e2e_steps, "s_per_step": sum(times) / len(times)}


def _quantiles(x, torch):
    """median, p90, p99 and max of a device tensor (float64)."""
    q = torch.quantile(x.float(), torch.tensor([0.5, 0.9, 0.99], device=x.device)).tolist() \
        if x.numel() <= 16_000_000 else [None] * 3
    return {"median": q[0], "p90": q[1], "p99": q[2], "max": float(x.max())}


def run_config4(ens, torch, stream, dev, m=1024, tuned=True):
    """1024 x 1024 Keller-Miksis grid, 64 periods, four solves: plain FP64 at
    tol 1e-10 and at 1e-8, the split-precision variant (FP32 with compensated
    sums, FP64 time and control) at 1e-8, the double-float variant at 1e-10.
    Speedups at equal tolerance and against the 1e-10 FP64 solve; per-system
    relative error of the per-period maxima (max over the 64 periods) against
    the FP64 solve at the same tolerance and at 1e-10.  Launch shapes from
    the autotuner (else the hand-measured ones)."""
    km = W.km(m, m, n_phases=64)
    ph = km["phys"]
    n = ph["pA1"].size
    phys_d = [torch.from_numpy(ph[k]).to(dev) for k in ("pA1", "f1", "pA2", "f2", "theta", "RE")]
    C = ens.ens_km_coefficients(*phys_d, km["liquid"], stream=stream)
    y0 = torch.from_numpy(km["y0"]).to(dev)
    stream.synchronize()
    res = {"systems": n}
    maxrows = {}
    # hand-measured shapes on this grid: FP64 26.6 s at 5-12 warps/SM; split precision 1.14 s at 24;
    # double-float 10.1 s at 16
    hand = {ens.ENS_FP64: (256, 1), ens.ENS_FP32_COMP: (256, 3), ens.ENS_FP32X2: (256, 2)}
    flops = {ens.ENS_FP64: (FLOPS_PER_KM_TRIAL, FP64_PEAK), ens.ENS_FP32_COMP: (FLOPS_FP32_PER_FP32C_TRIAL, FP32_PEAK),
             ens.ENS_FP32X2: (FLOPS_FP32_PER_DF_TRIAL, FP32_PEAK)}
    for name, prec, tl in (("fp64_tol1e-10", ens.ENS_FP64, 1e-10), ("fp64_tol1e-8", ens.ENS_FP64, 1e-8),
                           ("fp32c_tol1e-8", ens.ENS_FP32_COMP, 1e-8), ("fp32x2_tol1e-10", ens.ENS_FP32X2, 1e-10)):
        t = ens.make_tol(rtol=tl, atol=tl, dt0=1e-2, dt_min=1e-14, dt_max=1e-1, n_phases=64, prec=prec,
                         timeout_s=900.0)
        ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, n, C, y0, (0.0, 1.0), ens.ENS_RKCK45, t)
        try:
            ens.ens_set_launch(ctx, ens.make_launch(block=hand[prec][0], blocks_per_sm=hand[prec][1], cost_order=1))
            tune_s = None
            if tuned:
                t0 = time.perf_counter()
                ens.ens_autotune(ctx, stream)
                tune_s = time.perf_counter() - t0
            L = ens.ens_get_launch(ctx)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ens.ens_solve(ctx, stream)
            e1.record(stream)
            stream.synchronize()
            st = ens.ens_sync(ctx)
            kms = ens.ens_kernel_ms(ctx)
            nacc = ens.ens_read(ctx, ens.ENS_NSTEPS)
            nrej = ens.ens_read(ctx, ens.ENS_NREJ)
            acc = torch.empty((128, n), dtype=torch.float64, device=dev)
            ens.ens_read(ctx, ens.ENS_ACC, acc)
            maxrows[name] = acc[0::2].clone()
            del acc
        finally:
            ens.ens_destroy(ctx)
        ms = e0.elapsed_time(e1)
        trials = float(nacc.sum() + nrej.sum())
        fl, peak = flops[prec]
        res[name] = {"ms": ms, "kernel_ms": kms, "steps": float(nacc.sum()), "trials": trials,
                     "value": float(nacc.sum()) / (ms / 1e3), "unit": "system-steps/s", "status": st,
                     "launch": L.as_dict(), "tune_s": tune_s,
                     "frac": fl * trials / (kms / 1e3) / peak if fl else None}

    def rel(a, b):   # per system: max over periods of |a - b| / |b|
        return ((a - b).abs() / b.abs()).amax(dim=0)

    ref, ref8 = maxrows["fp64_tol1e-10"], maxrows["fp64_tol1e-8"]
    res["fp64_tol1e-8_vs_fp64_1e-10"] = _quantiles(rel(ref8, ref), torch)
    res["fp32c_vs_fp64_same_tol"] = _quantiles(rel(maxrows["fp32c_tol1e-8"], ref8), torch)
    res["fp32c_vs_fp64_1e-10"] = _quantiles(rel(maxrows["fp32c_tol1e-8"], ref), torch)
    d2 = rel(maxrows["fp32x2_tol1e-10"], ref)
    res["fp32x2_vs_fp64"] = _quantiles(d2, torch)
    res["fp32x2_vs_fp64"]["frac_below_1e-8"] = float((d2 < 1e-8).double().mean())
    res["speedup_fp32c_vs_fp64_same_tol"] = res["fp64_tol1e-8"]["ms"] / res["fp32c_tol1e-8"]["ms"]
    res["speedup_fp32c_vs_fp64_1e-10"] = res["fp64_tol1e-10"]["ms"] / res["fp32c_tol1e-8"]["ms"]
    res["speedup_fp32x2_vs_fp64"] = res["fp64_tol1e-10"]["ms"] / res["fp32x2_tol1e-10"]["ms"]
    del maxrows
    torch.cuda.empty_cache()
    return res


def run_screen(ens, torch, stream, dev, ctx, km, solve_ms, solve_steps, args):
    """Surrogate-screened scan: the headline solve's accessories train a
    4-member network; a held-out sample of the screening grid calibrates the
    fallback gate (spread > 0.05, or a steep predicted map) for an unflagged
    p99 error within the bound; the flagged points of the log grid are
    re-solved in FP64; a uniform sub-grid solved in FP64 validates the map
    and gives the measured FP64 cost."""
    from paper_2011_01740_gb300 import screen
    rows = ens.ens_acc_rows(ctx)
    n = km["phys"]["pA1"].size
    acc = torch.empty((rows, n), dtype=torch.float64, device=dev)
    ens.ens_read(ctx, ens.ENS_ACC, acc)
    x, y = screen.training_set_from_acc(ens, km, acc, rows // 2, rows // 4, dev, stream)
    r = screen.run(ens, screen_m=args.screen_m, n_phases=rows // 2, first_phase=rows // 4, threshold=0.05,
                   bound=args.screen_bound, calib_points=16384, val_stride=4, epochs=args.screen_epochs,
                   batch=args.screen_batch, lr=args.screen_lr, stream=stream, train=(x, y, solve_ms / 1e3, solve_steps),
                   fallback_launch=ens.ens_get_launch(ctx))
    r["screen_grid"] = [args.screen_m, args.screen_m]
    # screened scan throughput: grid points per second of screen + FP64 fallback
    r["value"] = r["screen_points"] / r["screened_total_s"]
    r["unit"] = "points/s"
    return r


def run_lyapunov(ens, torch, stream, dev, C_d, km, launch, n_phases=64, n_transient=32):
    """Largest Lyapunov exponent over the headline sweep: the Keller-Miksis
    tangent system, renormalised at every phase end on the device (Sec. 1,
    trajectory manipulation between phases), exponent = mean of the recorded
    per-phase log growths (phases 33-64) per unit tau."""
    n = km["phys"]["pA1"].size
    y0 = np.vstack([np.ones(n), np.zeros(n), np.ones(n), np.ones(n)])
    t = km["tol"]
    tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max, n_phases=n_phases,
                       n_transient=n_transient, timeout_s=900.0)
    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS_TANGENT, n, C_d, torch.from_numpy(y0).to(dev), (0.0, 1.0),
                         ens.ENS_RKCK45, tol)
    try:
        ens.ens_set_launch(ctx, launch)
        ens.ens_solve(ctx, stream)
        ens.ens_sync(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ens.ens_solve(ctx, stream)
        e1.record(stream)
        st = ens.ens_sync(ctx)
        ms = e0.elapsed_time(e1)
        acc = ens.ens_read(ctx, ens.ENS_ACC)
        nacc = ens.ens_read(ctx, ens.ENS_NSTEPS)
        kms = ens.ens_kernel_ms(ctx)
    finally:
        ens.ens_destroy(ctx)
    R = n_phases - n_transient
    lam = acc[2 * R:].mean(axis=0)                       # per unit tau (phase_len = 1)
    forced = km["phys"]["pA1"] > 0
    return {"ms": ms, "kernel_ms": kms, "status": st, "accepted_steps": float(nacc.sum()),
            "value": float(nacc.sum()) / (ms / 1e3), "unit": "system-steps/s",
            "chaotic_fraction": float(np.mean(lam[forced] > 0.0)),
            "lambda_quantiles": {q: float(np.percentile(lam[forced], q)) for q in (5, 50, 95)}}


def run_work_precision(ens, torch, stream, dev, m_f=16384):
    """Tolerance-error-work study of Sec. 4.2.2 on a full ensemble: p_A = 1.5 bar,
    m_f frequencies log-spaced over 20 kHz - 1 MHz, tau in [0, 2], both pairs
    at T = 1e-6 ... 1e-12; the global error E = |y1(2) - y1^E(2)| is taken
    against a Dormand-Prince run at T = 1e-14."""
    km = W.km(1, m_f, n_phases=1, pa_max=1.5e5)
    ph = km["phys"]
    ph["pA1"][:] = 1.5e5
    C = ens.ens_km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"], km["liquid"])
    launch = ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=160, blocks_per_sm=1, cost_order=1)

    def solve(solver, T):
        tol = ens.make_tol(rtol=T, atol=T, dt0=1e-2, dt_min=1e-14, dt_max=1e-1, timeout_s=600.0)
        ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, m_f, C, km["y0"], (0.0, 2.0), solver, tol)
        try:
            ens.ens_set_launch(ctx, launch)
            ens.ens_solve(ctx, stream)
            ens.ens_sync(ctx)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ens.ens_solve(ctx, stream)
            e1.record(stream)
            st = ens.ens_sync(ctx)
            return (ens.ens_read(ctx, ens.ENS_STATE)[0], float(ens.ens_read(ctx, ens.ENS_NRHS).sum()),
                    float(ens.ens_read(ctx, ens.ENS_NSTEPS).sum()), e0.elapsed_time(e1), st)
        finally:
            ens.ens_destroy(ctx)

    ref = solve(ens.ENS_DOPRI5, 1e-14)[0]
    out = {"systems": m_f, "reference": "Dormand-Prince, T = 1e-14"}
    for name, solver in (("cashkarp", ens.ENS_RKCK45), ("dopri5", ens.ENS_DOPRI5)):
        rows = []
        for k in (6, 8, 10, 12):
            y, nrhs, nacc, ms, st = solve(solver, 10.0 ** -k)
            E = np.abs(y - ref)
            rows.append({"tol": 10.0 ** -k, "status": st, "ms": ms, "rhs_per_system": nrhs / m_f,
                         "accepted_steps_per_s": nacc / (ms / 1e3),
                         "E_median": float(np.median(E)), "E_p90": float(np.percentile(E, 90)),
                         "E_max": float(E.max())})
        out[name] = rows
    return out


def run_dopri5(ens, torch, stream, dev, ck_ctx, C_d, y0_d, km, tol, launch, ck_ms):
    """The headline sweep with the Dormand-Prince pair (the solver of the
    paper's Julia runs, Sec. 4.2) on the same launch: throughput and the
    right-hand-side evaluations against the Cash-Karp run."""
    n = km["phys"]["pA1"].size
    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, n, C_d, y0_d, (0.0, 1.0), ens.ENS_DOPRI5, tol)
    try:
        ens.ens_set_launch(ctx, launch)
        ens.ens_solve(ctx, stream)                 # warm-up (also builds the graph)
        ens.ens_sync(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ens.ens_solve(ctx, stream)
        e1.record(stream)
        st = ens.ens_sync(ctx)
        ms = e0.elapsed_time(e1)
        nacc = ens.ens_read(ctx, ens.ENS_NSTEPS)
        nrej = ens.ens_read(ctx, ens.ENS_NREJ)
        nrhs = ens.ens_read(ctx, ens.ENS_NRHS)
        acc = ens.ens_read(ctx, ens.ENS_ACC)
    finally:
        ens.ens_destroy(ctx)
    ck_nrhs = ens.ens_read(ck_ctx, ens.ENS_NRHS)
    ck_acc = ens.ens_read(ck_ctx, ens.ENS_ACC)
    ck_nacc = ens.ens_read(ck_ctx, ens.ENS_NSTEPS)
    # per-period maxima of the two pairs on the non-chaotic systems: both meet
    # the same tolerance, so they agree to about the global error
    rel = np.abs(acc[0::2] - ck_acc[0::2]) / np.abs(ck_acc[0::2])
    per_sys = np.nanmax(rel, axis=0)
    return {"ms": ms, "status": st, "accepted_steps": float(nacc.sum()), "trials": float(nacc.sum() + nrej.sum()),
            "value": float(nacc.sum()) / (ms / 1e3), "unit": "system-steps/s",
            "rhs_evals": float(nrhs.sum()), "rhs_evals_cashkarp": float(ck_nrhs.sum()),
            "rhs_ratio_cashkarp_over_dopri5": float(ck_nrhs.sum() / nrhs.sum()),
            "accepted_steps_cashkarp": float(ck_nacc.sum()),
            "time_ratio_dopri5_over_cashkarp": ms / ck_ms,
            "acc_max_rel_diff_vs_cashkarp": {"median": float(np.median(per_sys)),
                                             "p90": float(np.percentile(per_sys, 90))}}


def _timed_km_solve(ens, torch, stream, dev, w, launch, n_transient=0, warm=False):
    """One Keller-Miksis phase-mode solve of workload w on the given launch:
    device time, counts and the recorded per-phase maxima."""
    ph = w["phys"]
    n = ph["pA1"].size
    phys_d = [torch.from_numpy(ph[k]).to(dev) for k in ("pA1", "f1", "pA2", "f2", "theta", "RE")]
    C = ens.ens_km_coefficients(*phys_d, w["liquid"], stream=stream)
    stream.synchronize()
    t = w["tol"]
    tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max, n_phases=t.n_phases,
                       n_transient=n_transient, timeout_s=900.0)
    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, n, C, torch.from_numpy(w["y0"]).to(dev), (0.0, 1.0),
                         ens.ENS_RKCK45, tol)
    try:
        ens.ens_set_launch(ctx, launch)
        if warm:
            ens.ens_solve(ctx, stream)
            ens.ens_sync(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ens.ens_solve(ctx, stream)
        e1.record(stream)
        st = ens.ens_sync(ctx)
        ms = e0.elapsed_time(e1)
        nacc = ens.ens_read(ctx, ens.ENS_NSTEPS)
        nrej = ens.ens_read(ctx, ens.ENS_NREJ)
        acc = ens.ens_read(ctx, ens.ENS_ACC)
        kms = ens.ens_kernel_ms(ctx)
    finally:
        ens.ens_destroy(ctx)
    return {"ms": ms, "kernel_ms": kms, "status": st, "systems": n, "accepted_steps": float(nacc.sum()),
            "trials": float(nacc.sum() + nrej.sum()), "value": float(nacc.sum()) / (ms / 1e3),
            "unit": "system-steps/s"}, acc


def run_frequency_response(ens, torch, stream, dev):
    """The paper's Keller-Miksis workload (Sec. 4.2): 46,080 frequencies at
    P_A1 = 1.5 bar, 1024 transient phases integrated and discarded, the
    maxima of the next 64 recorded; one solve, a persistent launch with
    longest-first claiming at 3 warps/SM."""
    w = W.km_frequency_response()
    # 46,080 systems of 787k trials on average: the longest ones bound the run,
    # and each warp's trials run fastest with few warps sharing the FP64 pipes
    # (measured: 3 warps/SM 35.8 s, 4: 39.1 s, 5: 49.0 s, 8: 74.3 s, 10: 92.5 s)
    res, acc = _timed_km_solve(ens, torch, stream, dev, w,
                               ens.make_launch(block=96, blocks_per_sm=1, cost_order=1), n_transient=w["n_transient"])
    y1max = acc[0::2].max(axis=0)
    res["phases"] = {"transient": w["n_transient"], "recorded": w["tol"].n_phases - w["n_transient"]}
    res["y1max_range"] = [float(y1max.min()), float(y1max.max())]
    res["launch"] = {"block": 96, "blocks_per_sm": 1, "cost_order": 1}
    return res


def run_dual_frequency(ens, torch, stream, dev, launch):
    """The 362 x 362 sweep with a second driving component (P_A2 = P_A1 / 2
    at f2 = 2 f1, theta = 0; 64 phases): the dual-frequency Keller-Miksis
    kernel on the headline launch."""
    res, _ = _timed_km_solve(ens, torch, stream, dev, W.km_dual(), launch, warm=True)
    res["forcing"] = {"pA2_over_pA1": 0.5, "f2_over_f1": 2.0, "theta": 0.0}
    return res


def run_fp32x2(ens, torch, stream, dev, ck_ctx, C_d, y0_d, km, tol, ck_ms):
    """The headline sweep in double-float arithmetic (ENS_FP32X2: pairs of
    floats on the FP32 pipes, time and forcing in FP64): time, speedup over
    the FP64 solve and the per-system difference of the per-period maxima
    from the FP64 solve's."""
    n = km["phys"]["pA1"].size
    t = km["tol"]
    tol2 = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                        n_phases=t.n_phases, phase_len=t.phase_len, prec=ens.ENS_FP32X2, timeout_s=900.0)
    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, n, C_d, y0_d, (0.0, 1.0), ens.ENS_RKCK45, tol2)
    try:
        # 7 warps/SM measured best (6: 1.80 s, 7: 1.79 s, 8: 1.97 s, 12: 2.71 s)
        ens.ens_set_launch(ctx, ens.make_launch(block=224, blocks_per_sm=1, cost_order=1))
        ens.ens_solve(ctx, stream)
        ens.ens_sync(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ens.ens_solve(ctx, stream)
        e1.record(stream)
        st = ens.ens_sync(ctx)
        ms = e0.elapsed_time(e1)
        nacc = ens.ens_read(ctx, ens.ENS_NSTEPS)
        nrej = ens.ens_read(ctx, ens.ENS_NREJ)
        acc = ens.ens_read(ctx, ens.ENS_ACC)
        kms = ens.ens_kernel_ms(ctx)
    finally:
        ens.ens_destroy(ctx)
    ref = ens.ens_read(ck_ctx, ens.ENS_ACC)
    rel = np.abs(acc[0::2] - ref[0::2]).max(axis=0) / np.abs(ref[0::2]).max(axis=0)
    return {"ms": ms, "kernel_ms": kms, "status": st, "accepted_steps": float(nacc.sum()),
            "trials": float(nacc.sum() + nrej.sum()), "value": float(nacc.sum()) / (ms / 1e3),
            "unit": "system-steps/s", "speedup_vs_fp64": ck_ms / ms,
            "launch": {"block": 224, "blocks_per_sm": 1, "cost_order": 1},
            "per_period_max_rel_diff_vs_fp64": {"median": float(np.median(rel)),
                                                "p90": float(np.percentile(rel, 90)),
                                                "frac_below_1e-8": float(np.mean(rel < 1e-8))}}


def run_secondary(ens, torch, stream, dev, tuned=True):
    """The other hot-path workloads, timed the same way (one launch each after
    a warm-up): RK4 peak-calibration x' = x^2 - p (Sec. 3), RK4 Lorenz
    (Sec. 4.1) at the configured 16,384 systems and over N up to the paper's
    768,000, and the relief valve with events (Sec. 4.3).  Launches from the
    autotuner (else the hand-measured ones)."""
    out = {}

    def timed(ctx, reps):
        ens.ens_solve(ctx, stream)
        ens.ens_sync(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ens.ens_solve(ctx, stream)
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps

    # x' = x^2 - p, 2^20 systems, 1000 steps: FP64 pipe calibration
    wl = W.x2p(1 << 20)
    ctx = ens.ens_create(ens.ENS_SYS_TOY_X2P, 1 << 20, wl["params"], wl["y0"], (0, 0), ens.ENS_RK4,
                         ens.make_tol(dt0=wl["dt"], n_steps=wl["nsteps"]))
    ens.ens_set_launch(ctx, ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=128))
    ms = timed(ctx, 5)
    ens.ens_destroy(ctx)
    sps = (1 << 20) * 1000 / (ms / 1e3)
    out["x2p_rk4_calibration"] = {"systems": 1 << 20, "ms": ms, "value": sps, "unit": "system-steps/s",
                                  "fp64_tflops": sps * FLOPS_PER_X2P_STEP / 1e12,
                                  "fp64_frac": sps * FLOPS_PER_X2P_STEP / FP64_PEAK}
    # Lorenz, 1000 steps: the configured 16,384 systems, and an N sweep up to
    # the paper's 768,000 (Sec. 4.1.2), each with its tuned launch
    sweep = {}
    for N in (16384, 65536, 262144, 768000):
        wl = W.lorenz(N)
        ctx = ens.ens_create(ens.ENS_SYS_LORENZ, N, wl["params"], wl["y0"], (0, 0), ens.ENS_RK4,
                             ens.make_tol(dt0=wl["dt"], n_steps=wl["nsteps"]))
        ens.ens_set_launch(ctx, ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=32))
        best = ens.ens_autotune(ctx, stream) if tuned else ens.ens_get_launch(ctx)
        table = _tune_table(ens, ctx) if tuned else None
        ms = timed(ctx, 20 if N <= 65536 else 5)
        ens.ens_destroy(ctx)
        sps = N * 1000 / (ms / 1e3)
        sweep[N] = {"ms": ms, "value": sps, "unit": "system-steps/s",
                    "fp64_frac": sps * FLOPS_PER_LORENZ_STEP / FP64_PEAK, "launch": best.as_dict(), "tune_table": table}
    out["lorenz_rk4_16384"] = sweep[16384]
    out["lorenz_rk4_n_sweep"] = sweep
    # relief valve, 262144 systems, t in [0, 1024], events
    wl = W.prv(262144)
    t = wl["tol"]
    tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                       event_tol=t.event_tol, acc_t_start=t.acc_t_start, timeout_s=900.0)
    ctx = ens.ens_create(ens.ENS_SYS_RELIEF_VALVE, 262144, wl["params"], wl["y0"], (t.t0, t.t1),
                         ens.ENS_RKCK45, tol)
    # hand-measured: 8 warps per SM (128: 19.0 s, 160/192: 18.1 s, 256: 18.0 s before the integer compares)
    ens.ens_set_launch(ctx, ens.make_launch(block=256, blocks_per_sm=1, use_graph=1, cost_order=1))
    tune_s = None
    if tuned:
        t0 = time.perf_counter()
        ens.ens_autotune(ctx, stream)
        tune_s = time.perf_counter() - t0
    L = ens.ens_get_launch(ctx)
    valve_table = _tune_table(ens, ctx) if tuned else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.ens_solve(ctx, stream)
    e1.record(stream)
    st = ens.ens_sync(ctx)
    ms = e0.elapsed_time(e1)
    kms = ens.ens_kernel_ms(ctx)
    nacc = ens.ens_read(ctx, ens.ENS_NSTEPS)
    nrej = ens.ens_read(ctx, ens.ENS_NREJ)
    acc64 = torch.empty((35, 262144), dtype=torch.float64, device=dev)
    ens.ens_read(ctx, ens.ENS_ACC, acc64)
    ens.ens_destroy(ctx)
    trials = float(nacc.sum() + nrej.sum())
    out["relief_valve_262144"] = {"ms": ms, "kernel_ms": kms, "status": st, "value": float(nacc.sum()) / (ms / 1e3),
                                  "unit": "system-steps/s", "trials": trials, "launch": L.as_dict(), "tune_s": tune_s,
                                  "tune_table": valve_table,
                                  "fp64_frac": (FLOPS_PER_VALVE_TRIAL * trials / (kms / 1e3) / FP64_PEAK
                                                if FLOPS_PER_VALVE_TRIAL else None),
                                  "fp64_form_frac": FLOPS_FP64_FORM_VALVE_TRIAL * trials / (kms / 1e3) / FP64_PEAK}
    # the same sweep in double-float arithmetic (state, stages, right-hand
    # side and controller as float pairs; time, events, impact law and
    # sticking in FP64): speedup, event counts and value rows against FP64
    tol2 = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                        event_tol=t.event_tol, acc_t_start=t.acc_t_start, timeout_s=900.0, prec=ens.ENS_FP32X2)
    ctx = ens.ens_create(ens.ENS_SYS_RELIEF_VALVE, 262144, wl["params"], wl["y0"], (t.t0, t.t1),
                         ens.ENS_RKCK45, tol2)
    ens.ens_set_launch(ctx, ens.make_launch(block=256, blocks_per_sm=1, use_graph=1, cost_order=1))
    tune2 = None
    if tuned:
        t0 = time.perf_counter()
        ens.ens_autotune(ctx, stream)
        tune2 = time.perf_counter() - t0
    L2 = ens.ens_get_launch(ctx)
    e0.record(stream)
    ens.ens_solve(ctx, stream)
    e1.record(stream)
    st2 = ens.ens_sync(ctx)
    ms2 = e0.elapsed_time(e1)
    kms2 = ens.ens_kernel_ms(ctx)
    nacc2 = ens.ens_read(ctx, ens.ENS_NSTEPS)
    nrej2 = ens.ens_read(ctx, ens.ENS_NREJ)
    acc2 = torch.empty((35, 262144), dtype=torch.float64, device=dev)
    ens.ens_read(ctx, ens.ENS_ACC, acc2)
    ens.ens_destroy(ctx)
    same_events = (acc2[33:35] == acc64[33:35]).all(dim=0)
    d = (acc2[:33] - acc64[:33]).abs()
    d = torch.where(torch.isnan(acc2[:33]) & torch.isnan(acc64[:33]), torch.zeros_like(d), d)
    rel = (d.amax(dim=0) / acc64[:33].abs().nan_to_num(0.0).amax(dim=0).clamp_min(1e-300))[same_events]
    q = _quantiles(rel, torch)
    trials2 = float(nacc2.sum() + nrej2.sum())
    out["relief_valve_262144"]["fp32x2"] = {
        "ms": ms2, "kernel_ms": kms2, "s": ms2 / 1e3, "status": st2, "value": float(nacc2.sum()) / (ms2 / 1e3),
        "speedup": ms / ms2, "launch": L2.as_dict(), "tune_s": tune2,
        "fp32_frac": FLOPS_FP32_PER_DF_VALVE_TRIAL * trials2 / (kms2 / 1e3) / FP32_PEAK,
        "same_event_counts": float(same_events.double().mean()),
        "value_rows_rel_diff_vs_fp64": q, "err_p99": q["p99"]}
    return out


# ---------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------

def _oracle_sample_solve(km, idx, nthreads=0):
    import oracle
    sub = W.take(km, idx)
    ph = sub["phys"]
    C = oracle.km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"],
                               oracle.liquid(**sub["liquid"]))
    t = sub["tol"]
    otol = oracle.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                           n_phases=t.n_phases, phase_len=t.phase_len, t0=t.t0)
    t0 = time.perf_counter()
    r = oracle.cashkarp_solve(oracle.KM, C, sub["y0"], otol, nthreads=nthreads)
    return float(r["nacc"].sum()), time.perf_counter() - t0


def cpu_baseline(km, seconds: float):
    """The oracle (plain C, all host cores) on a stratified sample of the same
    131,044 systems, sized to about `seconds` of CPU time."""
    import oracle
    n = km["phys"]["pA1"].size
    k = 256
    steps, el = _oracle_sample_solve(km, W.subsample(n, k))
    if el < seconds / 4:
        k = int(min(n, k * max(1.0, seconds / max(el, 1e-3))))
        steps, el = _oracle_sample_solve(km, W.subsample(n, k))
    # one host core, for comparison with the paper's single-core CPU runs
    s1, e1 = _oracle_sample_solve(km, W.subsample(n, 256), nthreads=1)
    # and the x' = x^2 - p RK4 calibration (21 flop per step, Sec. 3) on one core
    cal = W.x2p(4096)
    t0 = time.perf_counter()
    oracle.rk4_solve(oracle.X2P, cal["params"], cal["y0"], 0.0, cal["dt"], cal["nsteps"], nthreads=1)
    ec = time.perf_counter() - t0
    cal_sps = 4096 * cal["nsteps"] / ec
    return {"value": steps / el, "unit": "system-steps/s", "cores": oracle.max_threads(),
            "kind": "oracle", "sample": f"{k} of {n} systems (stratified, seed {W.SEED}), 64 periods",
            "seconds": el, "single_core_value": s1 / e1, "single_core_sample": "256 systems, 1 thread",
            "x2p_rk4_single_core": {"value": cal_sps, "unit": "system-steps/s", "gflops": cal_sps * 21 / 1e9,
                                    "sample": f"4096 systems x {cal['nsteps']} steps, 1 thread"}}


def run_reference(args):
    world, rank, local = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    km = km_slice(1, 0, n_phases=args.phases)
    n = km["phys"]["pA1"].size
    k = args.ref_systems
    idx = W.subsample(n, k)
    for _ in range(args.warmup):
        _oracle_sample_solve(km, W.subsample(n, min(k, 64)))
    tot_steps, tot_s = 0.0, 0.0
    for _ in range(args.steps):
        s, el = _oracle_sample_solve(km, idx)
        tot_steps += s
        tot_s += el
    value = tot_steps / tot_s
    cpu = {"value": value, "unit": "system-steps/s", "cores": oracle.max_threads(), "kind": "oracle",
           "sample": f"{k} of {n} systems (stratified, seed {W.SEED}) per step, 64 periods"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "system-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (deterministic parameter grid)",
            "config": {"workload": WORKLOAD, "systems": n, "sampled_systems_per_step": k},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "system-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile_case(case: str):
    """One small run of a workload (after one warm-up run) for ncu captures;
    prints the step counts that turn instruction counters into per-step
    figures."""
    import torch
    import paper_2011_01740_gb300 as ens
    torch.cuda.set_device(0)
    if case == "km":
        km = km_slice(1, 0, n_phases=2)
        idx = W.subsample(km["phys"]["pA1"].size, 4096)
        km = W.take(km, idx)
        ph = km["phys"]
        C = ens.ens_km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"],
                                    km["liquid"])
        t = km["tol"]
        tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                           n_phases=t.n_phases, phase_len=t.phase_len)
        ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0),
                             ens.ENS_RKCK45, tol)
        ens.ens_set_launch(ctx, ens.make_launch(block=128, blocks_per_sm=2, cost_order=0))
    elif case == "km_pow":
        # the 362 x 362 sweep with gamma = 1.33 (C10 = 3.99 is not 21/5): the
        # general-exponent kernel, whose right-hand side calls pow(); 2 periods
        km = km_slice(1, 0, n_phases=2)
        ph = km["phys"]
        liquid = dict(km["liquid"], gamma=1.33)
        C = ens.ens_km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"], liquid)
        t = km["tol"]
        tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                           n_phases=t.n_phases, phase_len=t.phase_len)
        ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0),
                             ens.ENS_RKCK45, tol)
        ens.ens_set_launch(ctx, ens.make_launch(block=160, blocks_per_sm=1, cost_order=0))
    elif case == "km_full64":
        # the benchmarked launch (all systems, 64 periods, longest-first claiming)
        km = km_slice(1, 0, n_phases=64)
        ph = km["phys"]
        C = ens.ens_km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"],
                                    km["liquid"])
        t = km["tol"]
        tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                           n_phases=t.n_phases, phase_len=t.phase_len)
        ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0),
                             ens.ENS_RKCK45, tol)
        ens.ens_set_launch(ctx, ens.make_launch(block=192, blocks_per_sm=1, cost_order=1))
    elif case == "km_full2":
        # all 131,044 systems, 2 periods: the instruction mix of the benchmarked kernel
        km = km_slice(1, 0, n_phases=2)
        ph = km["phys"]
        C = ens.ens_km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"],
                                    km["liquid"])
        t = km["tol"]
        tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                           n_phases=t.n_phases, phase_len=t.phase_len)
        ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0),
                             ens.ENS_RKCK45, tol)
        ens.ens_set_launch(ctx, ens.make_launch(block=160, blocks_per_sm=1, cost_order=0))
    elif case == "km_fp32c":
        km = km_slice(1, 0, n_phases=2)
        idx = W.subsample(km["phys"]["pA1"].size, 16384)
        km = W.take(km, idx)
        ph = km["phys"]
        C = ens.ens_km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"],
                                    km["liquid"])
        tol = ens.make_tol(rtol=1e-8, atol=1e-8, dt0=1e-2, dt_min=1e-14, dt_max=1e-1, n_phases=2,
                           prec=ens.ENS_FP32_COMP)
        ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0),
                             ens.ENS_RKCK45, tol)
        ens.ens_set_launch(ctx, ens.make_launch(block=256, blocks_per_sm=1, cost_order=0))
    elif case == "km_fp32x2":
        # 16,384 stratified systems of the 362 x 362 sweep, 2 periods, tol 1e-10, double-float
        km = km_slice(1, 0, n_phases=2)
        idx = W.subsample(km["phys"]["pA1"].size, 16384)
        km = W.take(km, idx)
        ph = km["phys"]
        C = ens.ens_km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"],
                                    km["liquid"])
        t = km["tol"]
        tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                           n_phases=t.n_phases, phase_len=t.phase_len, prec=ens.ENS_FP32X2)
        ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0),
                             ens.ENS_RKCK45, tol)
        ens.ens_set_launch(ctx, ens.make_launch(block=224, blocks_per_sm=1, cost_order=0))
    elif case in ("mlp_screen", "mlp_screen_mma"):
        import torch
        m = ens.ens_mlp_create(4, W.SEED)
        ens.ens_mlp_set_screen_impl(m, 0 if case == "mlp_screen_mma" else 1)
        pa, f = W.screen_grid(512)
        n = pa.size
        x = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        ens.ens_km_features(n, torch.from_numpy(pa).cuda(), torch.from_numpy(f).cuda(), W.KM_FEATURE_RANGE, x)
        outs = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
        for _ in range(2):
            ens.ens_mlp_screen(m, n, x, *outs)
        torch.cuda.synchronize()
        ens.ens_mlp_destroy(m)
        print(json.dumps({"case": case, "points": n, "members": 4,
                          "mac_per_point_member": 49664}), flush=True)
        return
    elif case == "mlp_train":
        # two epochs over 8,192 samples, batch 1024 (8 Adam steps per epoch):
        # the second epoch's launches are the ones to capture
        import torch
        x, y = W.mlp_batch(8192, seed=11)
        m = ens.ens_mlp_create(4, W.SEED)
        hist = ens.ens_mlp_train(m, 8192, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                                 ens.make_train_cfg(epochs=2, batch=1024, lr=2e-3), 4)
        torch.cuda.synchronize()
        ens.ens_mlp_destroy(m)
        print(json.dumps({"case": case, "samples": 8192, "batch": 1024, "members": 4, "epochs": 2,
                          "flop_per_launch_per_kernel": 3 * 2 * 128 * 128 * 1024 * 4,
                          "loss": [float(hist[0].mean()), float(hist[-1].mean())]}), flush=True)
        return
    elif case in ("prv", "prv_df"):
        wl = W.prv(8192, t1=64.0)
        t = wl["tol"]
        tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                           event_tol=t.event_tol, acc_t_start=t.acc_t_start,
                           prec=ens.ENS_FP32X2 if case == "prv_df" else ens.ENS_FP64)
        ctx = ens.ens_create(ens.ENS_SYS_RELIEF_VALVE, 8192, wl["params"], wl["y0"], (t.t0, t.t1),
                             ens.ENS_RKCK45, tol)
    elif case in ("x2p", "lorenz"):
        wl = W.x2p(1 << 20) if case == "x2p" else W.lorenz(16384)
        sysid = ens.ENS_SYS_TOY_X2P if case == "x2p" else ens.ENS_SYS_LORENZ
        ctx = ens.ens_create(sysid, wl["params"].shape[1], wl["params"], wl["y0"], (0, 0), ens.ENS_RK4,
                             ens.make_tol(dt0=wl["dt"], n_steps=wl["nsteps"]))
        ens.ens_set_launch(ctx, ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=128))
    else:
        raise SystemExit(f"unknown profile case {case}")
    for _ in range(2):
        ens.ens_solve(ctx)
        st = ens.ens_sync(ctx)
    nacc = ens.ens_read(ctx, ens.ENS_NSTEPS)
    nrej = ens.ens_read(ctx, ens.ENS_NREJ)
    print(json.dumps({"case": case, "systems": int(nacc.size), "status": int(st),
                      "accepted": int(nacc.sum()), "rejected": int(nrej.sum()),
                      "trials": int(nacc.sum() + nrej.sum())}), flush=True)
    ens.ens_destroy(ctx)


def run_probe(case: str):
    """Timing probes behind the launch-shape reasoning (one JSON line each):
    pipe_sharing -- copies of the 362 x 362 sweep's longest Keller-Miksis
    system at controlled occupancy (1 to 8 warps on one SM, 4 and 5 warps on
    every SM; 16 periods), the main kernel's time per trial;
    trial_distribution -- trials per system of the full sweep (64 periods) and
    of its one-phase pilot: quantiles, the share of the longest systems, the
    pilot's rank correlation with the full count."""
    import torch
    import paper_2011_01740_gb300 as ens
    torch.cuda.set_device(0)
    km = km_slice(1, 0, n_phases=64)
    ph = km["phys"]
    t = km["tol"]
    C = ens.ens_km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"], km["liquid"])

    def solve(Cs, y0, nph, launch):
        tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max, n_phases=nph,
                           timeout_s=900.0)
        ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, Cs.shape[1], Cs, y0, (0.0, 1.0), ens.ENS_RKCK45, tol)
        try:
            ens.ens_set_launch(ctx, launch)
            ens.ens_solve(ctx)
            assert ens.ens_sync(ctx) == ens.ENS_OK
            ens.ens_solve(ctx)
            assert ens.ens_sync(ctx) == ens.ENS_OK
            trials = ens.ens_read(ctx, ens.ENS_NSTEPS) + ens.ens_read(ctx, ens.ENS_NREJ)
            return ens.ens_kernel_ms(ctx), trials
        finally:
            ens.ens_destroy(ctx)

    if case == "trial_distribution":
        _, full = solve(C, km["y0"], 64, ens.make_launch(block=160, blocks_per_sm=1, cost_order=1))
        _, pilot = solve(C, km["y0"], 1, ens.make_launch(block=160, blocks_per_sm=1, cost_order=0))
        srt = np.sort(full)[::-1]
        rank = lambda a: np.argsort(np.argsort(a))
        print(json.dumps({"probe": case, "systems": int(full.size), "trials": int(full.sum()),
                          "mean": float(full.mean()), "max": int(full.max()),
                          "quantiles": {q: float(np.percentile(full, q)) for q in (50, 90, 99, 99.9)},
                          "top_k_min_and_share": {k: [int(srt[k - 1]), float(srt[:k].sum() / full.sum())]
                                                  for k in (10, 100, 1000, 10000)},
                          "pilot_rank_correlation": float(np.corrcoef(rank(full), rank(pilot))[0, 1])}), flush=True)
        return
    if case != "pipe_sharing":
        raise SystemExit(f"unknown probe {case}")
    _, full = solve(C, km["y0"], 64, ens.make_launch(block=160, blocks_per_sm=1, cost_order=1))
    i = int(np.argmax(full))            # the sweep's longest system
    PL = ens.ENS_LAUNCH_PLAIN
    rows = []
    for label, n, block in (("1 warp, 1 lane", 1, 32), ("1 warp, 32 lanes", 32, 32), ("2 warps", 64, 64),
                            ("4 warps, one per sub-partition", 128, 128), ("5 warps", 160, 160),
                            ("8 warps, two per sub-partition", 256, 256), ("4 warps on every SM", 128 * 152, 128),
                            ("5 warps on every SM", 160 * 152, 160)):
        Cn = np.repeat(C[:, i:i + 1], n, axis=1)
        y0 = np.repeat(km["y0"][:, i:i + 1], n, axis=1)
        ms, tr = solve(Cn, y0, 16, ens.make_launch(mode=PL, block=block))
        rows.append({"case": label, "systems": n, "block": block, "ms": ms, "trials": int(tr[0]),
                     "us_per_trial": 1e3 * ms / float(tr[0])})
    print(json.dumps({"probe": case, "system": i, "pA": float(ph["pA1"][i]), "f": float(ph["f1"][i]),
                      "periods": 16, "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile", default=None,
                    help="run one small case for ncu (km, km_full64, km_full2, km_pow, km_fp32c, km_fp32x2, mlp_screen, "
                         "mlp_screen_mma, mlp_train, prv, prv_df, x2p, lorenz)")
    ap.add_argument("--probe", default=None, help="timing probe (pipe_sharing, trial_distribution)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--phases", type=int, default=64)
    ap.add_argument("--block", type=int, default=192)
    ap.add_argument("--bps", type=int, default=1)
    ap.add_argument("--cost-order", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-systems", type=int, default=1024)
    ap.add_argument("--quick", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--screen-m", type=int, default=4096, help="screening grid side (4096 x 4096 = 16.8M points)")
    # training length and batch of the surrogate: 2,400 epochs of 8,192 samples (10 s) leave 1.6 % of the
    # 4096^2 grid to the FP64 fallback at the p99 bound; 150 epochs of 1,024 (1.9 s) left 16 %
    ap.add_argument("--screen-epochs", type=int, default=2400)
    ap.add_argument("--screen-batch", type=int, default=8192)
    ap.add_argument("--screen-lr", type=float, default=6e-3)
    ap.add_argument("--screen-bound", type=float, default=0.05,
                    help="unflagged p99 |ln r error| the screening gate is calibrated for")
    ap.add_argument("--no-tune", action="store_true", help="hand-measured launch shapes instead of ens_autotune")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.profile:
        run_profile_case(args.profile)
        return
    if args.probe:
        run_probe(args.probe)
        return
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
