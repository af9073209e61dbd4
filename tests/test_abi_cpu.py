"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point of include/ens.h; argument validation fails cleanly; the host
planner (Keller-Miksis coefficients) agrees with the oracle's own derivation."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "ens.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ens_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def ens():
    import paper_2011_01740_gb300 as ens
    ens.lib()
    return ens


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("ens_create", "ens_solve", "ens_sync", "ens_read", "ens_last_error", "ens_destroy",
                 "ens_set_inputs", "ens_set_launch", "ens_autotune", "ens_km_coefficients"):
        assert must in names


def test_library_exports_every_declared_symbol(ens):
    L = ens.lib()
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert "sm_103a" in ens.ens_version()


def test_python_binding_has_the_same_names(ens):
    for n in _declared_functions():
        assert hasattr(ens, n), n


def test_create_rejects_bad_arguments_without_touching_a_device(ens):
    tol = ens.make_tol(dt0=0.01, n_steps=10)
    with pytest.raises(ens.EnsError) as e:
        ens.ens_create(ens.ENS_SYS_LORENZ, -1, np.zeros((3, 1)), np.zeros((3, 1)), (0, 0), ens.ENS_RK4, tol)
    assert e.value.status == ens.ENS_EINVAL
    with pytest.raises(ens.EnsError) as e:
        ens.ens_create(7, 1, np.zeros((3, 1)), np.zeros((3, 1)), (0, 0), ens.ENS_RK4, tol)
    assert e.value.status == ens.ENS_EINVAL
    with pytest.raises(ens.EnsError) as e:   # RK4 cannot run the impacting valve
        ens.ens_create(ens.ENS_SYS_RELIEF_VALVE, 1, np.zeros((5, 1)), np.zeros((3, 1)), (0, 1),
                       ens.ENS_RK4, tol)
    assert e.value.status == ens.ENS_ENOTSUP
    bad = ens.make_tol(rtol=-1.0)
    with pytest.raises(ens.EnsError) as e:
        ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, 1, np.zeros((13, 1)), np.zeros((2, 1)), (0, 1),
                       ens.ENS_RKCK45, bad)
    assert e.value.status == ens.ENS_EINVAL
    assert "rtol" in ens.ens_last_error(None)


def test_transient_phase_count_is_validated(ens):
    """n_transient: 0 <= n_transient < n_phases in phase mode, 0 otherwise;
    checked before any device work."""
    C = np.zeros((13, 1))
    y0 = np.array([[1.0], [0.0]])
    for nt, nph in ((4, 4), (-1, 4), (1, 0)):
        with pytest.raises(ens.EnsError) as e:
            ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, 1, C, y0, (0.0, 1.0), ens.ENS_RKCK45,
                           ens.make_tol(n_phases=nph, n_transient=nt))
        assert e.value.status == ens.ENS_EINVAL
        assert "n_transient" in ens.ens_last_error(None)


def test_reduced_precision_variants_are_limited_to_their_kernels(ens):
    """ENS_FP32_COMP exists for the Keller-Miksis phase mode with Cash-Karp,
    ENS_FP32X2 for that and for the relief valve's event mode with Cash-Karp;
    everything else is refused before any device work."""
    C = np.zeros((13, 1))
    y0 = np.array([[1.0], [0.0]])
    for prec in (ens.ENS_FP32_COMP, ens.ENS_FP32X2):
        for solver, nph in ((ens.ENS_DOPRI5, 2), (ens.ENS_RKCK45, 0)):
            with pytest.raises(ens.EnsError) as e:
                ens.ens_create(ens.ENS_SYS_KELLER_MIKSIS, 1, C, y0, (0.0, 1.0), solver,
                               ens.make_tol(n_phases=nph, prec=prec))
            assert e.value.status == ens.ENS_ENOTSUP
    for prec, solver in ((ens.ENS_FP32_COMP, ens.ENS_RKCK45), (ens.ENS_FP32X2, ens.ENS_DOPRI5)):
        with pytest.raises(ens.EnsError) as e:
            ens.ens_create(ens.ENS_SYS_RELIEF_VALVE, 1, np.zeros((5, 1)), np.zeros((3, 1)), (0.0, 1.0),
                           solver, ens.make_tol(event_tol=1e-6, prec=prec))
        assert e.value.status == ens.ENS_ENOTSUP
    with pytest.raises(ens.EnsError) as e:   # Lorenz has no reduced-precision kernel
        ens.ens_create(ens.ENS_SYS_LORENZ, 1, np.zeros((3, 1)), np.zeros((3, 1)), (0.0, 1.0), ens.ENS_RKCK45,
                       ens.make_tol(prec=ens.ENS_FP32X2))
    assert e.value.status == ens.ENS_ENOTSUP


def test_null_context_calls_are_harmless(ens):
    L = ens.lib()
    assert L.ens_solve(None, None) == ens.ENS_EINVAL
    assert L.ens_sync(None) == ens.ENS_EINVAL
    assert L.ens_acc_rows(None) == 0
    ms = ctypes.c_double(1.0)
    assert L.ens_kernel_ms(None, ctypes.byref(ms)) == ens.ENS_EINVAL
    L.ens_destroy(None)


def test_host_planner_matches_oracle_coefficients(ens):
    import oracle
    from paper_2011_01740_gb300 import workloads as W
    rng = np.random.default_rng(5)
    n = 500
    pA1, pA2 = rng.uniform(0, 2e5, n), rng.uniform(0, 1e5, n)
    f1, f2 = rng.uniform(2e4, 1e6, n), rng.uniform(0, 2e6, n)
    th, RE = rng.uniform(0, 6.28, n), rng.uniform(1e-6, 1e-4, n)
    C = ens.ens_km_coefficients(pA1, f1, pA2, f2, th, RE, W.WATER_25C)
    Co = oracle.km_coefficients(pA1, f1, pA2, f2, th, RE, oracle.liquid(**W.WATER_25C))
    np.testing.assert_allclose(C, Co, rtol=4e-15, atol=0)


def test_noalloc_validates_like_create_before_any_device_work(ens):
    """ens_solve_noalloc applies ens_create's tolerance checks (a negative rtol
    with a positive atol is refused) and its own cap on n, all before it
    touches a device."""
    z = np.zeros(1)
    outs = [z] * 8
    bad = ens.make_tol(rtol=-1.0, atol=1e-10, n_phases=2)
    with pytest.raises(ens.EnsError) as e:
        ens.ens_solve_noalloc(ens.ENS_SYS_KELLER_MIKSIS, 1, z, z, (0.0, 1.0), bad, *outs)
    assert e.value.status == ens.ENS_EINVAL
    assert "rtol" in str(e.value)
    with pytest.raises(ens.EnsError) as e:
        ens.ens_solve_noalloc(ens.ENS_SYS_KELLER_MIKSIS, (1 << 20) + 1, z, z, (0.0, 1.0),
                              ens.make_tol(n_phases=2), *outs)
    assert e.value.status == ens.ENS_EINVAL and "1048576" in str(e.value)
    with pytest.raises(ens.EnsError) as e:   # the valve runs in event mode only
        ens.ens_solve_noalloc(ens.ENS_SYS_RELIEF_VALVE, 1, z, z, (0.0, 1.0),
                              ens.make_tol(n_phases=2, event_tol=1e-6), *outs)
    assert e.value.status == ens.ENS_EINVAL
