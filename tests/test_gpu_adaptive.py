"""GPU parity of the adaptive Cash-Karp path: Keller-Miksis phase mode
(Sec. 4.2) and the pressure relief valve with events (Sec. 4.3), through the
C ABI, against the CPU oracle.

Adaptive runs amplify rounding differences through the step sequence (an
accept / reject decision that flips moves every later step point, and the
per-period maximum is sampled at step points).  The comparison therefore
runs on the well-conditioned systems, those whose oracle accessories move by
less than 1e-9 when the initial state is perturbed by 1e-14 relative; there
the GPU must match to 1e-8 relative.  The excluded fraction is bounded.
"""
import numpy as np
import pytest

import oracle
import paper_2011_01740_gb300 as ens
from paper_2011_01740_gb300 import workloads as W
from gpu_helpers import (ens_tol_from, km_coeffs_lib, km_coeffs_oracle, oracle_tol_from, rel_err,
                         solve_gpu)

pytestmark = pytest.mark.gpu

ACC_TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ens.lib()


def _well_conditioned(sys, params, y0, otol, deltas=(1e-14, -3e-15), rows=None):
    """Oracle run plus the systems whose accessories move by less than 1e-9
    under each relative perturbation of the initial state in `deltas`."""
    a = oracle.cashkarp_solve(sys, params, y0, otol)
    sel = slice(None) if rows is None else rows
    well = a["status"] == 0
    for d in deltas:
        b = oracle.cashkarp_solve(sys, params, np.asarray(y0) * (1 + d), otol)
        well &= (rel_err(b["acc"][sel], a["acc"][sel]) < 1e-9) & (b["status"] == 0)
    return a, well


# ---------------------------------------------------------------------------
# Keller-Miksis
# ---------------------------------------------------------------------------

def _km_gpu(km, launch=None, n_phases=None, **tolkw):
    C = km_coeffs_lib(km["phys"], km["liquid"])
    t = km["tol"]
    tol = ens_tol_from(t, **({"n_phases": n_phases} if n_phases else {}), **tolkw)
    return solve_gpu(ens.ENS_SYS_KELLER_MIKSIS, C, km["y0"], (t.t0, t.t1), ens.ENS_RKCK45, tol,
                     launch=launch)


def test_km_small_grid_parity():
    km = W.km(19, 23, n_phases=4)          # 437 systems: 3 full blocks + a ragged tail
    g = _km_gpu(km)
    Co = km_coeffs_oracle(km["phys"], km["liquid"])
    r, well = _well_conditioned(oracle.KM, Co, km["y0"], oracle_tol_from(km["tol"]))
    assert g["sync"] == ens.ENS_OK and np.all(g["status"] == 0)
    assert well.mean() > 0.9
    err = rel_err(g["acc"], r["acc"])
    assert np.all(err[well] < ACC_TOL), err[well].max()
    assert np.all(rel_err(g["y"], r["y"])[well] < 1e-7)
    # same step sequence on the well-conditioned systems
    d = np.abs(g["nacc"] - r["nacc"]) / r["nacc"]
    assert np.median(d[well]) == 0.0 and d[well].max() <= 0.05
    assert np.all(g["nrhs"] == 6 * (g["nacc"] + g["nrej"]) - g["nrej"])


def test_km_full_grid_sampled_parity():
    """131,044 systems (362 x 362 p_A x f grid), 64 periods, tol 1e-10: the
    benchmarked launch, checked on a stratified sample of 192 systems."""
    km = W.km()
    g = _km_gpu(km)
    n = km["y0"].shape[1]
    assert g["sync"] == ens.ENS_OK and np.all(g["status"] == 0)
    idx = W.subsample(n, 192)
    sub = W.take(km, idx)
    Co = km_coeffs_oracle(sub["phys"], sub["liquid"])
    r, well = _well_conditioned(oracle.KM, Co, sub["y0"], oracle_tol_from(km["tol"]))
    assert well.mean() > 0.75, well.mean()
    err = rel_err(g["acc"][:, idx], r["acc"])
    assert np.all(err[well] < ACC_TOL), (err[well].max(), idx[well][np.argmax(err[well])])
    # every system: accessories are physical radii, finite and ordered
    acc = g["acc"]
    assert np.all(np.isfinite(acc)) and np.all(acc[0::2] >= acc[1::2]) and np.all(acc[1::2] > 0)
    # the unforced row p_A = 0 stays at the equilibrium radius
    assert np.abs(acc[:, :362] - 1.0).max() < 1e-8


def test_km_launch_modes_and_graph_replay_are_bitwise_identical():
    km = W.km(13, 29, n_phases=3)
    ref = _km_gpu(km, launch=ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=64))
    for L in (ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=128, blocks_per_sm=1),
              ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=64, blocks_per_sm=4, use_graph=1),
              ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=128, blocks_per_sm=2, cost_order=1)):
        g = _km_gpu(km, launch=L)
        for k in ("y", "acc", "nacc", "nrej", "nrhs", "status", "dt"):
            assert np.array_equal(g[k], ref[k], equal_nan=True), (k, L.as_dict())


def test_persistent_refill_solves_every_system_as_the_plain_launch():
    """30,000 systems on 4,864 to 34,048 persistent lanes: lanes refill from
    the claim counter many times over (longest-first or in index order), and
    every system comes out bitwise as in the plain one-thread-per-system launch."""
    km = W.km(150, 200, n_phases=2)
    ref = _km_gpu(km, launch=ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=128))
    for L in (ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=160, blocks_per_sm=1, cost_order=1),
              ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=224, blocks_per_sm=1, cost_order=0),
              ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=32, blocks_per_sm=1, cost_order=1)):
        g = _km_gpu(km, launch=L)
        assert np.all(g["nacc"] > 0)
        for k in ("y", "acc", "nacc", "nrej", "nrhs", "status", "dt"):
            assert np.array_equal(g[k], ref[k], equal_nan=True), (k, L.as_dict())


@pytest.mark.parametrize("block", [160, 192, 224])
@pytest.mark.parametrize("m", [(19, 23), (3, 40), (150, 200)])
def test_first_claims_by_subpartition_cover_every_system_once(block, m):
    """Persistent, longest-first, one block per SM: the first claims are ranked
    by sub-partition (lanes of warps that own theirs first), later ones
    continue from the counter.  With 120, 437 and 30,000 systems (fewer
    systems than the unshared lanes, between them and all lanes, and many
    refills) every system is solved once and comes out bitwise as in the
    plain launch."""
    km = W.km(*m, n_phases=2)
    ref = _km_gpu(km, launch=ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=128))
    g = _km_gpu(km, launch=ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=block, blocks_per_sm=1,
                                           cost_order=1))
    assert g["sync"] == ens.ENS_OK and np.all(g["nacc"] > 0)
    for k in ("y", "acc", "nacc", "nrej", "nrhs", "status", "dt"):
        assert np.array_equal(g[k], ref[k], equal_nan=True), k


@pytest.mark.parametrize("prec", [ens.ENS_FP64, ens.ENS_FP32_COMP])
def test_transient_phases_are_integrated_but_not_recorded(prec):
    """n_transient = 5 of 8 phases: the recorded rows are the last 3 phases of
    the run that records all 8, bitwise, in both precisions."""
    km = W.km(11, 13, n_phases=8)
    kw = dict(prec=prec) if prec == ens.ENS_FP64 else dict(prec=prec, rtol=1e-8, atol=1e-8)
    full = _km_gpu(km, **kw)
    part = _km_gpu(km, n_transient=5, **kw)
    assert full["acc"].shape[0] == 16 and part["acc"].shape[0] == 6
    assert np.array_equal(part["acc"], full["acc"][10:], equal_nan=True)
    for k in ("y", "nacc", "nrej", "status"):
        assert np.array_equal(part[k], full[k], equal_nan=True), k


def test_transient_phases_match_the_oracle():
    """A paper-style run, transient phases then recorded ones (Sec. 4.2), on a
    small grid: the recorded rows against the oracle's full record."""
    km = W.km(6, 7, n_phases=12)
    g = _km_gpu(km, n_transient=8)
    Co = km_coeffs_oracle(km["phys"], km["liquid"])
    r, well = _well_conditioned(oracle.KM, Co, km["y0"], oracle_tol_from(km["tol"]))
    assert g["sync"] == ens.ENS_OK and well.mean() > 0.75
    err = rel_err(g["acc"], r["acc"][16:])
    assert np.all(err[well] < ACC_TOL), err[well].max()


def test_km_graph_replays_and_set_inputs():
    km = W.km(9, 11, n_phases=2)
    C = km_coeffs_lib(km["phys"], km["liquid"])
    tol = ens_tol_from(km["tol"])
    n = C.shape[1]
    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, n, C, km["y0"], (0.0, 1.0), ens.ENS_RKCK45, tol)
    try:
        ens.ens_set_launch(ctx, ens.make_launch(use_graph=1))
        outs = []
        for _ in range(3):
            ens.ens_solve(ctx)
            assert ens.ens_sync(ctx) == ens.ENS_OK
            outs.append(ens.ens_read(ctx, ens.ENS_ACC))
        assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
        # new inputs through the same context (and graph)
        y0b = km["y0"].copy()
        y0b[0] = 1.05
        ens.ens_set_inputs(ctx, None, y0b)
        ens.ens_solve(ctx)
        ens.ens_sync(ctx)
        accb = ens.ens_read(ctx, ens.ENS_ACC)
    finally:
        ens.ens_destroy(ctx)
    Co = km_coeffs_oracle(km["phys"], km["liquid"])
    r = oracle.cashkarp_solve(oracle.KM, Co, y0b, oracle_tol_from(km["tol"]))
    assert np.median(rel_err(accb, r["acc"])) < 1e-9


def test_km_device_planner_matches_host_planner():
    import torch
    km = W.km(31, 37)
    ph = km["phys"]
    host = km_coeffs_lib(ph, km["liquid"])
    dev = ens.ens_km_coefficients(*[torch.from_numpy(ph[k]).cuda() for k in
                                    ("pA1", "f1", "pA2", "f2", "theta", "RE")], km["liquid"])
    torch.cuda.synchronize()
    np.testing.assert_allclose(dev.cpu().numpy(), host, rtol=4e-16, atol=0)


def test_km_dual_frequency_parity():
    """Second driving component (P_A2, f2, theta != 0) with the omega2 form of C8."""
    rng = np.random.default_rng(3)
    n = 150
    phys = dict(pA1=rng.uniform(0.2e5, 1.5e5, n), f1=rng.uniform(1e5, 8e5, n),
                pA2=rng.uniform(0.1e5, 0.8e5, n), f2=rng.uniform(1e5, 1.5e6, n),
                theta=rng.uniform(0, 6.28, n), RE=np.full(n, 10e-6))
    km = dict(phys=phys, liquid=W.WATER_25C, y0=np.stack([np.ones(n), np.zeros(n)]),
              tol=W.Tolerances(n_phases=3))
    g = _km_gpu(km)
    Co = km_coeffs_oracle(phys, W.WATER_25C)
    r, well = _well_conditioned(oracle.KM, Co, km["y0"], oracle_tol_from(km["tol"]))
    assert well.mean() > 0.8
    assert np.all(rel_err(g["acc"], r["acc"])[well] < ACC_TOL)


def test_km_status_words():
    km = W.km(3, 4, n_phases=2)
    g = _km_gpu(km, max_steps=5)
    big = g["nacc"] + g["nrej"]
    assert np.all((g["status"] & ens.ENS_SYS_MAX_STEPS) > 0)
    assert np.all(big == 5)
    assert np.all(np.isnan(g["acc"][2:]))           # phase 1 never completed
    assert g["sync"] == ens.ENS_ESYSTEM
    # an unreachable tolerance underflows the step size (the driven systems;
    # the unforced ones sit at their fixed point up to rounding)
    g = _km_gpu(km, rtol=1e-30, atol=1e-30, dt_min=1e-6)
    forced = km["phys"]["pA1"] > 0
    assert np.all((g["status"][forced] & ens.ENS_SYS_DT_UNDERFLOW) > 0)
    # the wall-clock budget stops the solve and is reported, not waited out
    g = _km_gpu(W.km(20, 20, n_phases=64), timeout_s=1e-6)
    assert np.all((g["status"] & ens.ENS_SYS_TIMEOUT) > 0)
    assert g["sync"] == ens.ENS_ETIMEOUT


# ---------------------------------------------------------------------------
# pressure relief valve
# ---------------------------------------------------------------------------

def _prv(n, t1, q_min=0.2, q_max=10.0):
    return W.prv(n, q_min=q_min, q_max=q_max, t1=t1)


def _prv_gpu(wl, launch=None, **tolkw):
    t = wl["tol"]
    tol = ens_tol_from(t, **tolkw)
    return solve_gpu(ens.ENS_SYS_RELIEF_VALVE, wl["params"], wl["y0"], (t.t0, t.t1), ens.ENS_RKCK45,
                     tol, launch=launch)


def _prv_compare(g, r, well, idx=None):
    gi = (lambda a: a) if idx is None else (lambda a: a[..., idx])
    acc = gi(g["acc"])
    # counts of maxima and impacts agree exactly on the well-conditioned systems
    assert np.array_equal(acc[33][well], r["acc"][33][well])
    assert np.array_equal(acc[34][well], r["acc"][34][well])
    err = rel_err(acc[:33], r["acc"][:33])
    assert np.all(err[well] < ACC_TOL), err[well].max()
    assert np.all(rel_err(gi(g["y"]), r["y"])[well] < 1e-7)


def test_prv_small_parity():
    wl = _prv(300, 64.0)
    g = _prv_gpu(wl)
    r, well = _well_conditioned(oracle.PRV, wl["params"], wl["y0"], oracle_tol_from(wl["tol"]),
                                 rows=slice(0, 33))
    assert g["sync"] == ens.ENS_OK and np.all(g["status"] == 0)
    assert well.mean() > 0.75, well.mean()
    _prv_compare(g, r, well)
    assert np.all(g["t"] == 64.0)


def test_prv_full_sweep_sampled_parity():
    """262,144 valves, t in [0, 1024]: the benchmarked launch, on a sample."""
    wl = _prv(262144, 1024.0)
    g = _prv_gpu(wl)
    bad = np.nonzero(g["status"])[0]
    assert bad.size == 0, (np.bincount(g["status"]), wl["params"][0][bad[:20]].tolist(),
                           g["nacc"][bad[:5]].tolist(), g["t"][bad[:5]].tolist())
    assert g["sync"] == ens.ENS_OK
    idx = W.subsample(262144, 96)
    sub = W.take(wl, idx)
    r, well = _well_conditioned(oracle.PRV, sub["params"], sub["y0"], oracle_tol_from(wl["tol"]),
                                 rows=slice(0, 33))
    assert well.mean() > 0.5, well.mean()
    _prv_compare(g, r, well, idx)
    # every valve: impacting below q ~ 7.5 (Sec. 4.3), pressure non-negative
    q = wl["params"][0]
    ymin = g["acc"][32]
    assert np.mean(ymin[q < 7.0] == 0.0) > 0.95 and np.all(ymin[q > 8.0] > 0.0)
    assert np.all(g["y"][2] >= 0.0)


def test_prv_grazing_impact_matches_oracle():
    """A recorded valve state (q = 7.5393) that dips about 1e-5 below the seat
    under a strong opening force: the event location must converge on the
    GPU (no EVENT_NO_CONVERGE), with one impact and the oracle's end state,
    from three initial step proposals."""
    params = np.array([[7.5392987796736906], [1.25], [10.0], [20.0], [0.8]])
    y0 = np.array([[0.0013698420381308958], [-0.3162497537150412], [45.746744783524875]])
    for dt0 in (0.0085, 0.008889370476683223, 0.0107):
        kw = dict(rtol=1e-10, atol=1e-10, dt0=dt0, dt_min=1e-14, dt_max=1.0, event_tol=1e-6, acc_t_start=0.0)
        g = solve_gpu(ens.ENS_SYS_RELIEF_VALVE, params, y0, (0.0, 0.05), ens.ENS_RKCK45, ens.make_tol(**kw))
        r = oracle.cashkarp_solve(oracle.PRV, params, y0, oracle.make_tol(t0=0.0, t1=0.05, **kw))
        assert g["status"][0] == 0 and r["status"][0] == 0
        assert g["acc"][34, 0] == 1 and r["acc"][34, 0] == 1
        assert np.all(rel_err(g["y"], r["y"]) < 1e-7), (g["y"][:, 0], r["y"][:, 0])


def test_prv_launch_modes_bitwise_identical():
    wl = _prv(200, 32.0)
    ref = _prv_gpu(wl, launch=ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=128))
    g = _prv_gpu(wl, launch=ens.make_launch(mode=ens.ENS_LAUNCH_PERSISTENT, block=64, blocks_per_sm=1,
                                            cost_order=1))
    for k in ("y", "acc", "nacc", "nrej", "status"):
        assert np.array_equal(g[k], ref[k], equal_nan=True), k


@pytest.mark.parametrize("use_graph", [0, 1])
def test_kernel_ms_times_the_main_launch(use_graph):
    """ens_kernel_ms: positive, and below the whole solve (which adds the
    one-phase pilot and the claim-order sort), with and without graph replay."""
    import torch
    km = W.km(24, 24, n_phases=4)
    C = km_coeffs_lib(km["phys"], km["liquid"])
    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0),
                         ens.ENS_RKCK45, ens_tol_from(km["tol"]))
    try:
        with pytest.raises(ens.EnsError):
            ens.ens_kernel_ms(ctx)                      # nothing enqueued yet
        ens.ens_set_launch(ctx, ens.make_launch(block=160, blocks_per_sm=1, use_graph=use_graph, cost_order=1))
        s = torch.cuda.Stream()
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            ens.ens_solve(ctx, s)
            e1.record(s)
            assert ens.ens_sync(ctx) == ens.ENS_OK
            s.synchronize()
            k = ens.ens_kernel_ms(ctx)
            assert 0.0 < k <= e0.elapsed_time(e1) * 1.001, (k, e0.elapsed_time(e1))
    finally:
        ens.ens_destroy(ctx)


def test_autotune_of_the_adaptive_solve():
    """The tuner times persistent launches of 3-24 warps per SM with
    longest-first claiming, the best residency without it, a plain launch and
    two systems per thread at 6 and 8 warps per SM, on a shortened horizon of
    every system (1/8 of 16 phases), times the two fastest again on twice
    that horizon, keeps the faster of those, and leaves results unchanged:
    the claim order and the launch shape never change what a system
    computes."""
    km = W.km(24, 20, n_phases=16)
    C = km_coeffs_lib(km["phys"], km["liquid"])
    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0),
                         ens.ENS_RKCK45, ens_tol_from(km["tol"]))
    try:
        ens.ens_solve(ctx)
        assert ens.ens_sync(ctx) == ens.ENS_OK
        ref = {w: ens.ens_read(ctx, w) for w in (ens.ENS_ACC, ens.ENS_STATE, ens.ENS_NSTEPS)}
        best = ens.ens_autotune(ctx)
        rows = ens.ens_autotune_table(ctx)
        # 13 candidates on 1/8 of the horizon, then the two fastest again on 1/4
        assert len(rows) == 15
        assert all(r["horizon_frac"] == 0.125 for r in rows[:13])
        assert all(r["horizon_frac"] == 0.25 for r in rows[13:])
        first = sorted(rows[:13], key=lambda r: r["ms"])[:2]
        assert [r["launch"] for r in rows[13:]] == [r["launch"] for r in first]
        rows, confirm = rows[:13], rows[13:]
        persistent = [r for r in rows if r["launch"]["mode"] == ens.ENS_LAUNCH_PERSISTENT]
        warps = lambda rs: {r["launch"]["block"] // 32 * r["launch"]["blocks_per_sm"] for r in rs}
        assert warps(r for r in persistent if r["launch"]["systems_per_thread"] == 1) == {3, 4, 5, 6, 7, 8, 12, 16, 24}
        assert warps(r for r in persistent if r["launch"]["systems_per_thread"] == 2) == {6, 8}
        assert any(r["launch"]["mode"] == ens.ENS_LAUNCH_PLAIN for r in rows)
        assert any(r["launch"]["cost_order"] == 0 for r in persistent)
        fastest = min(confirm, key=lambda r: r["ms"])["launch"]
        assert (fastest["mode"], fastest["block"], fastest["blocks_per_sm"], fastest["cost_order"],
                fastest["systems_per_thread"]) == \
            (best.mode, best.block, best.blocks_per_sm, best.cost_order, max(1, best.systems_per_thread))
        ens.ens_solve(ctx)
        assert ens.ens_sync(ctx) == ens.ENS_OK
        for w, v in ref.items():
            assert np.array_equal(ens.ens_read(ctx, w), v)
        # a second call returns the cached choice and table
        again = ens.ens_autotune(ctx)
        assert (again.block, again.blocks_per_sm) == (best.block, best.blocks_per_sm)
        assert len(ens.ens_autotune_table(ctx)) == len(rows) + len(confirm)
    finally:
        ens.ens_destroy(ctx)


_ALL_OUT = ("y", "acc", "status", "nacc", "nrej", "nrhs", "t", "dt")


@pytest.mark.parametrize("block,bps,cost_order,m,tolkw", [
    (128, 2, 1, (19, 23), {}),                          # 437 systems, ragged against 2 x 128 slots a lane pair
    (96, 2, 0, (19, 23), {"n_transient": 2}),           # transient phases, counter order
    (64, 1, 1, (1, 5), {}),                             # 5 systems: most slots never get one
    (128, 2, 1, (19, 23), {"max_steps": 150}),          # budget runs out mid-phase: NaN rows, status
])
def test_two_systems_per_thread_give_the_same_bits(block, bps, cost_order, m, tolkw):
    """Two systems per thread in the persistent phase-mode kernel: every output
    equals that of one system per thread bit for bit (each slot's step
    sequence is that of a lane of its own), with ragged ends, slots that never
    claim a system, transient phases and systems retired by the step budget."""
    km = W.km(*m, n_phases=6)
    one = _km_gpu(km, launch=ens.make_launch(block=128, blocks_per_sm=2, cost_order=cost_order), **tolkw)
    two = _km_gpu(km, launch=ens.make_launch(block=block, blocks_per_sm=bps, cost_order=cost_order,
                                             systems_per_thread=2), **tolkw)
    assert two["launch"]["systems_per_thread"] == 2
    assert one["sync"] == two["sync"]
    if "max_steps" in tolkw:
        assert np.any(one["status"] != 0) and np.any(np.isnan(one["acc"]))
    else:
        assert one["sync"] == ens.ENS_OK and np.all(one["status"] == 0)
    for k in _ALL_OUT:
        assert np.array_equal(one[k], two[k], equal_nan=True), k


def test_systems_per_thread_outside_the_kernel_that_has_it_are_refused():
    """Two systems per thread exist for the FP64 Cash-Karp phase mode of the
    Keller-Miksis model with one frequency and exponent 21/5, persistent, at
    most 128 threads a block; everything else is refused with ENS_ENOTSUP:
    when the launch is set, or, for a second driving frequency (a parameter
    property), when the solve is enqueued."""
    km = W.km(4, 4, n_phases=2)
    C = km_coeffs_lib(km["phys"], km["liquid"])
    tol = ens_tol_from(km["tol"])

    def refused(ctx, **kw):
        with pytest.raises(ens.EnsError) as e:
            ens.ens_set_launch(ctx, ens.make_launch(**kw))
        assert e.value.status == ens.ENS_ENOTSUP
        assert ens.ens_get_launch(ctx).systems_per_thread in (0, 1)

    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0), ens.ENS_RKCK45, tol)
    try:
        refused(ctx, block=128, blocks_per_sm=1, systems_per_thread=4)
        refused(ctx, block=256, blocks_per_sm=1, systems_per_thread=2)
        refused(ctx, mode=ens.ENS_LAUNCH_PLAIN, block=128, systems_per_thread=2)
        ens.ens_set_launch(ctx, ens.make_launch(block=128, blocks_per_sm=1, systems_per_thread=2))
        assert ens.ens_get_launch(ctx).systems_per_thread == 2
    finally:
        ens.ens_destroy(ctx)
    for solver, prec in ((ens.ENS_DOPRI5, ens.ENS_FP64), (ens.ENS_RKCK45, ens.ENS_FP32X2)):
        ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C.shape[1], C, km["y0"], (0.0, 1.0), solver,
                             ens_tol_from(km["tol"], prec=prec))
        try:
            refused(ctx, block=128, blocks_per_sm=1, systems_per_thread=2)
        finally:
            ens.ens_destroy(ctx)
    # a second driving frequency: accepted as a launch, refused by the solve
    phys = dict(km["phys"])
    phys["pA2"] = np.full(16, 2.0e4)
    phys["f2"] = np.full(16, 5.0e4)
    C2 = km_coeffs_lib(phys, km["liquid"])
    ctx = ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, C2.shape[1], C2, km["y0"], (0.0, 1.0), ens.ENS_RKCK45, tol)
    try:
        ens.ens_set_launch(ctx, ens.make_launch(block=128, blocks_per_sm=1, systems_per_thread=2))
        with pytest.raises(ens.EnsError) as e:
            ens.ens_solve(ctx)
        assert e.value.status == ens.ENS_ENOTSUP
    finally:
        ens.ens_destroy(ctx)
