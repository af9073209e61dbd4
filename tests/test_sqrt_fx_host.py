"""Host checks of the integer-pipe square root (csrc/sqrt_fx.cuh), built for
the CPU with g++, against 60-digit arithmetic (mpmath) and exact squares.

The claim under test: one fixed-point binomial step from a float seed leaves
the result within half an ulp plus 2^-58 relative of sqrt(x), for normal and
subnormal x of any exponent and for seeds off by up to 2^-19; exact for
perfect squares; +-0, +infinity, negative x and NaN handled as IEEE sqrt."""
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
    out = str(tmp_path_factory.mktemp("sqrtfx") / "sqrt_fx_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", f"-I{CSRC}",
                    os.path.join(HERE, "sqrt_fx_host.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    L.sqrt_fx_seed.argtypes = [ctypes.c_int64, P, ctypes.c_double, P]
    return L


def _run(lib, x, seed_rel=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    if seed_rel is None:
        lib.sqrt_fx_n(x.size, x.ctypes.data_as(P), out.ctypes.data_as(P))
    else:
        lib.sqrt_fx_seed(x.size, x.ctypes.data_as(P), float(seed_rel), out.ctypes.data_as(P))
    return out


def _check(x, got):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    for v, g in zip(x, got):
        e = mp.sqrt(mp.mpf(float(v)))
        ulp = float(np.spacing(float(e)))
        err = float(abs(mp.mpf(float(g)) - e))
        assert err <= 0.5 * ulp + 2.0 ** -58 * float(e), (v, g, err / ulp)


def test_random_arguments_within_the_bound(lib):
    rng = np.random.default_rng(13)
    x = np.concatenate([rng.uniform(0.0, 30.0, 3000), 10.0 ** rng.uniform(-300, 300, 2000),
                        rng.uniform(1.0, 4.0, 1000)])
    _check(x, _run(lib, x))


def test_subnormals_and_extremes(lib):
    x = np.array([5e-324, 1e-310, 2.0 ** -1074 * 12345, 2.0 ** -1022, np.nextafter(2.0 ** -1022, 0),
                  np.finfo(np.float64).max, 2.0 ** 1023])
    _check(x, _run(lib, x))


def test_perfect_squares_are_exact(lib):
    k = np.concatenate([np.arange(1, 5000), 2.0 ** np.arange(-500, 500, 7), [94906265.0]])
    got = _run(lib, k * k)
    assert np.array_equal(got, k)


def test_the_refinement_tolerates_seed_errors(lib):
    rng = np.random.default_rng(14)
    x = np.concatenate([rng.uniform(0.01, 30.0, 1000), 10.0 ** rng.uniform(-20, 20, 500)])
    for rel in (2.0 ** -19, -(2.0 ** -19)):
        _check(x, _run(lib, x, seed_rel=rel))


def test_special_values(lib):
    got = _run(lib, np.array([0.0, -0.0, np.inf, -1.0, -np.inf, np.nan, -5e-324]))
    assert got[0] == 0.0 and not np.signbit(got[0])
    assert got[1] == 0.0 and np.signbit(got[1])
    assert got[2] == np.inf
    assert np.all(np.isnan(got[3:]))
