"""Host checks of the integer-pipe x^(-1/5) (csrc/fifth_root_fx.cuh), built
for the CPU with g++, against 50-digit arithmetic (mpmath).

The claim under test: one fixed-point third-order step from a float seed
leaves a relative error below 2^-56 before the final rounding, so the result
is the correctly rounded double except near rounding boundaries (here: within
half an ulp plus 2^-56 relative), for positive normal x of any exponent, and
for seeds off by up to 2^-19 (the hardware seed has about 22 correct bits);
exact at powers of 32; NaN for x <= 0, NaN and infinity.  The polytropic
power x^(-21/5) built on the same fixed-point root stays within 1.5 ulp."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2011_01740_gb300", "csrc")
P = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("rootfx") / "fifth_root_fx_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", f"-I{CSRC}",
                    os.path.join(HERE, "fifth_root_fx_host.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    L.fifth_root_fx_seed.argtypes = [ctypes.c_int64, P, ctypes.c_double, P]
    L.pow_m21_5_fx_n.argtypes = [ctypes.c_int64, P, P]
    return L


def _run(lib, x, seed_rel=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    if seed_rel is None:
        lib.fifth_root_fx(x.size, x.ctypes.data_as(P), out.ctypes.data_as(P))
    else:
        lib.fifth_root_fx_seed(x.size, x.ctypes.data_as(P), float(seed_rel), out.ctypes.data_as(P))
    return out


def _check(x, got):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    worst = 0.0
    for v, g in zip(x, got):
        e = mp.power(mp.mpf(float(v)), mp.mpf(-1) / 5)
        ulp = float(np.spacing(float(e)))
        err = float(abs(mp.mpf(float(g)) - e))
        assert err <= 0.5 * ulp + 2.0 ** -56 * float(e), (v, g, err / float(e))
        worst = max(worst, err / ulp)
    return worst


def test_random_arguments_are_correctly_rounded_to_the_bound(lib):
    rng = np.random.default_rng(7)
    x = np.concatenate([10.0 ** rng.uniform(-30, 30, 3000), rng.uniform(0.01, 10.0, 2000),
                        10.0 ** rng.uniform(-300, 300, 500)])
    # half an ulp plus 2^-56 relative: at most 0.5 + 2^-56 / 2^-53 ulp
    assert _check(x, _run(lib, x)) < 0.625


def test_every_exponent_residue_and_the_extremes(lib):
    # e = 5 q + k for k = 0..4 and q of both signs, and the ends of the normal range
    x = np.array([m * 2.0 ** e for e in range(-30, 31) for m in (1.0, 1.37, 1.9999999)]
                 + [2.0 ** -1022, 1.5 * 2.0 ** -1022, np.nextafter(np.inf, 0), 2.0 ** 1023])
    _check(x, _run(lib, x))


def test_powers_of_32_are_exact(lib):
    q = np.arange(-40, 41)
    x = 32.0 ** q
    got = _run(lib, x)
    assert np.array_equal(got, 2.0 ** (-q.astype(np.float64)))
    assert _run(lib, np.array([1.0]))[0] == 1.0


def test_the_refinement_tolerates_seed_errors(lib):
    rng = np.random.default_rng(8)
    x = np.concatenate([rng.uniform(0.01, 10.0, 1000), 10.0 ** rng.uniform(-10, 10, 500)])
    for rel in (2.0 ** -19, -(2.0 ** -19), 2.0 ** -21):
        _check(x, _run(lib, x, seed_rel=rel))


def test_non_positive_and_non_finite_give_nan(lib):
    got = _run(lib, np.array([0.0, -0.0, -1.0, -1e-300, np.nan, np.inf, -np.inf]))
    assert np.all(np.isnan(got))


def _pow(lib, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lib.pow_m21_5_fx_n(x.size, x.ctypes.data_as(P), out.ctypes.data_as(P))
    return out


def test_polytropic_power_within_one_and_a_half_ulp(lib):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.uniform(0.001, 10.0, 3000), 10.0 ** rng.uniform(-60, 60, 1000),
                        [1.0, 2.0, 0.5, 1.5, np.nextafter(2.0, 0.0), np.nextafter(32.0, 0.0)]])
    got = _pow(lib, x)
    for v, g in zip(x, got):
        e = mp.power(mp.mpf(float(v)), mp.mpf(-21) / 5)
        ulp = float(np.spacing(float(e)))
        assert float(abs(mp.mpf(float(g)) - e)) <= 1.5 * ulp, (v, g)
    # powers of 32 exactly; outside the normal range 0 and infinity; NaN for x <= 0
    q = np.arange(-40, 41)
    assert np.array_equal(_pow(lib, 32.0 ** q), 2.0 ** (-21.0 * q))
    assert np.array_equal(_pow(lib, np.array([1e200, 1e-200])), np.array([0.0, np.inf]))
    assert np.all(np.isnan(_pow(lib, np.array([0.0, -2.0, np.nan, np.inf]))))
