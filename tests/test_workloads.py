"""The synthetic workload recipes (paper_2011_01740_gb300/workloads.py)
against the sweeps the paper describes: grids, fixed parameters, ordering,
and the determinism of the seeded parts."""
import numpy as np

from paper_2011_01740_gb300 import workloads as W


def test_grids_are_inclusive_and_logarithmic():
    g = W.linspace(0.1, 1.0, 10)
    assert g[0] == 0.1 and g[-1] == 1.0 and np.allclose(np.diff(g), 0.1)
    f = W.logspace(2e4, 1e6, 5)
    assert f[0] == 2e4 and np.isclose(f[-1], 1e6)
    np.testing.assert_allclose(f[1:] / f[:-1], (1e6 / 2e4) ** 0.25)


def test_keller_miksis_sweep_is_pa_by_f_with_f_fastest():
    w = W.km(4, 3, n_phases=64)
    ph = w["phys"]
    assert ph["pA1"].size == 12
    np.testing.assert_array_equal(ph["pA1"].reshape(4, 3)[:, 0], W.linspace(0.0, 2e5, 4))
    np.testing.assert_array_equal(ph["f1"].reshape(4, 3)[0], W.logspace(2e4, 1e6, 3))
    assert np.all(ph["pA2"] == 0) and np.all(ph["RE"] == 10e-6)
    assert np.array_equal(w["y0"], np.stack([np.ones(12), np.zeros(12)]))
    assert w["tol"].rtol == w["tol"].atol == 1e-10 and w["tol"].n_phases == 64


def test_frequency_response_is_the_papers_run():
    w = W.km_frequency_response()
    ph = w["phys"]
    assert ph["f1"].size == 46080
    assert np.all(ph["pA1"] == 1.5e5) and np.all(ph["pA2"] == 0) and np.all(ph["theta"] == 0)
    assert ph["f1"][0] == 2e4 and np.isclose(ph["f1"][-1], 1e6) and np.all(np.diff(ph["f1"]) > 0)
    assert w["n_transient"] == 1024 and w["tol"].n_phases == 1024 + 64


def test_dual_frequency_sweep_adds_the_second_component():
    base, dual = W.km(5, 6), W.km_dual(5, 6)
    for k in ("pA1", "f1", "RE"):
        np.testing.assert_array_equal(dual["phys"][k], base["phys"][k])
    np.testing.assert_array_equal(dual["phys"]["pA2"], 0.5 * base["phys"]["pA1"])
    np.testing.assert_array_equal(dual["phys"]["f2"], 2.0 * base["phys"]["f1"])


def test_relief_valve_and_lorenz_sweeps():
    v = W.prv(1000)
    assert v["params"].shape == (5, 1000)
    np.testing.assert_array_equal(v["params"][0], W.linspace(0.2, 10.0, 1000))
    assert np.all(v["params"][1:, 0] == [1.25, 10.0, 20.0, 0.8])
    assert v["tol"].t1 == 1024.0 and v["tol"].acc_t_start == 512.0 and v["tol"].event_tol == 1e-6
    lo = W.lorenz(100)
    np.testing.assert_array_equal(lo["params"][0], W.linspace(0.0, 21.0, 100))
    assert np.all(lo["params"][1] == 10.0) and np.allclose(lo["params"][2], 8.0 / 3.0)


def test_stratified_subsample_is_deterministic_and_covers_every_stratum():
    a, b = W.subsample(131044, 4096), W.subsample(131044, 4096)
    assert np.array_equal(a, b) and a.size == 4096 and np.all(np.diff(a) > 0)
    edges = np.linspace(0, 131044, 65).astype(np.int64)
    counts = np.histogram(a, bins=edges)[0]
    assert np.all(counts == 64)
    assert not np.array_equal(a, W.subsample(131044, 4096, seed=W.SEED + 1))
