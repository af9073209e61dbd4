"""GPU parity of the fixed-step RK4 path (Sec. 3 example, Sec. 4.1 Lorenz)
against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_2011_01740_gb300 as ens
from paper_2011_01740_gb300 import workloads as W
from gpu_helpers import rel_err, rk4_amplification, rk4_tolerance, solve_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ens.lib()


def _rk4(sys, wl, prec=ens.ENS_FP64, nsteps=None, launch=None):
    nsteps = wl["nsteps"] if nsteps is None else nsteps
    tol = ens.make_tol(dt0=wl["dt"], n_steps=nsteps, prec=prec)
    return solve_gpu(sys, wl["params"], wl["y0"], (wl["t0"], 0.0), ens.ENS_RK4, tol, launch=launch)


@pytest.mark.parametrize("n", [421, 16384])
def test_lorenz_strict_is_bit_identical_to_oracle(n):
    """Uncontracted FP64 in the oracle's operation order: identical bits."""
    wl = W.lorenz(n)
    g = _rk4(ens.ENS_SYS_LORENZ, wl, prec=ens.ENS_FP64_STRICT)
    yo, st = oracle.rk4_solve(oracle.LORENZ, wl["params"], wl["y0"], 0.0, wl["dt"], wl["nsteps"])
    assert g["sync"] == ens.ENS_OK
    assert np.array_equal(g["y"], yo)
    assert np.all(g["status"] == 0) and np.all(g["nacc"] == 1000) and np.all(g["nrhs"] == 4000)


@pytest.mark.parametrize("n", [421, 16384])
def test_lorenz_fast_matches_oracle_within_conditioned_bound(n):
    """FMA kernel (the benchmarked configuration) vs the oracle: within the
    derived bound max(1e-12, 8 N eps A) for every system (A: the oracle-measured
    growth of a relative perturbation; up to 1e5 in the transient chaos near
    rho = 21); most systems within 1e-12 outright."""
    wl = W.lorenz(n)
    g = _rk4(ens.ENS_SYS_LORENZ, wl)
    yo, A = rk4_amplification(ens.ENS_SYS_LORENZ, wl["params"], wl["y0"], wl["dt"], wl["nsteps"])
    err = rel_err(g["y"], yo)
    tol = rk4_tolerance(A, wl["nsteps"])
    assert np.all(err <= tol), (err / tol).max()
    within = (err <= 1e-12).mean()
    print(f"rk4 fma vs oracle: {within:.4f} of systems within 1e-12, max err {err.max():.2e}, "
          f"max err / bound {(err / tol).max():.3f}")
    assert within > 0.8
    np.testing.assert_array_equal(g["t"], np.full(n, 10.0))


def test_x2p_strict_and_fast():
    wl = W.x2p(1 << 16)
    gs = _rk4(ens.ENS_SYS_TOY_X2P, wl, prec=ens.ENS_FP64_STRICT)
    gf = _rk4(ens.ENS_SYS_TOY_X2P, wl)
    yo, _ = oracle.rk4_solve(oracle.X2P, wl["params"], wl["y0"], 0.0, wl["dt"], wl["nsteps"])
    assert np.array_equal(gs["y"], yo)
    assert rel_err(gf["y"], yo).max() < 1e-12


def test_x2p_full_size_sampled():
    """The 2^20-system calibration workload, checked on a stratified sample."""
    wl = W.x2p(1 << 20)
    g = _rk4(ens.ENS_SYS_TOY_X2P, wl)
    idx = W.subsample(1 << 20, 4096)
    sub = W.take(wl, idx)
    yo, _ = oracle.rk4_solve(oracle.X2P, sub["params"], sub["y0"], 0.0, wl["dt"], wl["nsteps"])
    assert rel_err(g["y"][:, idx], yo).max() < 1e-12


@pytest.mark.parametrize("block", [32, 64, 128, 256])
def test_launch_shapes_do_not_change_results(block):
    wl = W.lorenz(1000)
    ref = _rk4(ens.ENS_SYS_LORENZ, wl)
    g = _rk4(ens.ENS_SYS_LORENZ, wl, launch=ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=block))
    assert np.array_equal(ref["y"], g["y"])


def test_edge_sizes_and_nonfinite_status():
    for n in (1, 31, 33):
        wl = W.lorenz(n)
        g = _rk4(ens.ENS_SYS_LORENZ, wl, nsteps=50)
        yo, _ = oracle.rk4_solve(oracle.LORENZ, wl["params"], wl["y0"], 0.0, wl["dt"], 50)
        assert rel_err(g["y"], yo).max() < 1e-13
    # empty ensemble
    tol = ens.make_tol(dt0=0.01, n_steps=10)
    ctx = ens.ens_create(ens.ENS_SYS_LORENZ, 0, np.zeros((3, 0)), np.zeros((3, 0)), (0, 0), ens.ENS_RK4, tol)
    ens.ens_solve(ctx)
    assert ens.ens_sync(ctx) == ens.ENS_OK
    ens.ens_destroy(ctx)
    # x' = x^2 - p blows up from x0 = 2 with p = 0.1: reported, not hidden
    p = np.array([[0.1, 0.5]])
    y0 = np.array([[2.0, -0.5]])
    tol = ens.make_tol(dt0=0.01, n_steps=1000)
    g = solve_gpu(ens.ENS_SYS_TOY_X2P, p, y0, (0.0, 0.0), ens.ENS_RK4, tol)
    assert g["status"][0] & ens.ENS_SYS_NONFINITE and g["status"][1] == 0
    assert g["sync"] == ens.ENS_ESYSTEM


def test_device_inputs_and_destinations():
    import torch
    wl = W.lorenz(777)
    tol = ens.make_tol(dt0=wl["dt"], n_steps=100)
    P = torch.from_numpy(wl["params"]).cuda()
    Y = torch.from_numpy(wl["y0"]).cuda()
    ctx = ens.ens_create(ens.ENS_SYS_LORENZ, 777, P, Y, (0.0, 0.0), ens.ENS_RK4, tol)
    try:
        s = torch.cuda.Stream()
        ens.ens_solve(ctx, s)
        ens.ens_sync(ctx)
        dst = torch.empty((3, 777), dtype=torch.float64, device="cuda")
        ens.ens_read(ctx, ens.ENS_STATE, dst)
    finally:
        ens.ens_destroy(ctx)
    yo, _ = oracle.rk4_solve(oracle.LORENZ, wl["params"], wl["y0"], 0.0, wl["dt"], 100)
    assert rel_err(dst.cpu().numpy(), yo).max() < 1e-12


@pytest.mark.parametrize("prec", [ens.ENS_FP64, ens.ENS_FP64_STRICT])
@pytest.mark.parametrize("spt,block", [(2, 64), (4, 32), (4, 128)])
def test_systems_per_thread_gives_the_same_bits(prec, spt, block):
    """Two or four systems interleaved per thread run each system's steps
    with the arithmetic of one system per thread: every output is bitwise the
    same, including the ragged end of the ensemble (1,001 systems do not fill
    the last block's slots), and the strict flavour still equals the oracle."""
    wl = W.lorenz(1001)
    ref = _rk4(ens.ENS_SYS_LORENZ, wl, prec=prec, nsteps=300,
               launch=ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=32))
    got = _rk4(ens.ENS_SYS_LORENZ, wl, prec=prec, nsteps=300,
               launch=ens.make_launch(mode=ens.ENS_LAUNCH_PLAIN, block=block, systems_per_thread=spt))
    assert got["sync"] == ens.ENS_OK
    for k in ("y", "status", "nacc", "nrhs"):
        assert np.array_equal(got[k], ref[k]), k
    if prec == ens.ENS_FP64_STRICT:
        yo, _ = oracle.rk4_solve(oracle.LORENZ, wl["params"], wl["y0"], 0.0, wl["dt"], 300)
        assert np.array_equal(got["y"], yo)


def test_autotune_of_rk4_searches_systems_per_thread():
    """The tuner times block sizes x systems per thread on whole solves, keeps
    the fastest, and the tuned solve gives the untuned solve's bits."""
    wl = W.lorenz(4096)
    tol = ens.make_tol(dt0=wl["dt"], n_steps=200)
    ctx = ens.ens_create(ens.ENS_SYS_LORENZ, 4096, wl["params"], wl["y0"], (0.0, 0.0), ens.ENS_RK4, tol)
    try:
        ens.ens_solve(ctx)
        ens.ens_sync(ctx)
        ref = ens.ens_read(ctx, ens.ENS_STATE)
        best = ens.ens_autotune(ctx)
        rows = ens.ens_autotune_table(ctx)
        assert len(rows) == 12
        assert {r["launch"]["systems_per_thread"] for r in rows} == {1, 2, 4}
        fastest = min(rows, key=lambda r: r["ms"])
        assert fastest["launch"]["block"] == best.block
        assert fastest["launch"]["systems_per_thread"] == max(1, best.systems_per_thread)
        assert ens.ens_get_launch(ctx).block == best.block
        ens.ens_solve(ctx)
        assert ens.ens_sync(ctx) == ens.ENS_OK
        assert np.array_equal(ens.ens_read(ctx, ens.ENS_STATE), ref)
    finally:
        ens.ens_destroy(ctx)
