"""Host checks of the integer-pipe reciprocal (csrc/rcp_fx.cuh), built for
the CPU with g++, against exact rationals.

The claim under test: one fixed-point cubic Newton step from a float seed
leaves a relative error below 2^-57 before the final rounding, so the result
is within half an ulp plus 2^-57 relative of 1/d, for normal d of either sign
with |d| < 2^1022 and for seeds off by up to 2^-22; exact at powers of two;
NaN for zero, subnormal, infinite, NaN and too large d."""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

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
    out = str(tmp_path_factory.mktemp("rcpfx") / "rcp_fx_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", f"-I{CSRC}",
                    os.path.join(HERE, "rcp_fx_host.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    L.rcp_fx_seed.argtypes = [ctypes.c_int64, P, ctypes.c_double, P]
    return L


def _run(lib, d, seed_rel=None):
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.empty_like(d)
    if seed_rel is None:
        lib.rcp_fx_n(d.size, d.ctypes.data_as(P), out.ctypes.data_as(P))
    else:
        lib.rcp_fx_seed(d.size, d.ctypes.data_as(P), float(seed_rel), out.ctypes.data_as(P))
    return out


def _check(d, got):
    worst = 0.0
    for v, g in zip(d, got):
        e = 1 / Fraction(float(v))
        ulp = Fraction(float(np.spacing(abs(float(e)))))
        err = abs(Fraction(float(g)) - e)
        assert err <= ulp / 2 + abs(e) / 2 ** 57, (v, g)
        worst = max(worst, float(err / ulp))
    return worst


def test_random_arguments_within_the_bound(lib):
    rng = np.random.default_rng(9)
    d = rng.choice([-1.0, 1.0], 6000) * np.concatenate([10.0 ** rng.uniform(-30, 30, 3000),
                                                        rng.uniform(0.001, 10.0, 2500),
                                                        10.0 ** rng.uniform(-300, 300, 500)])
    assert _check(d, _run(lib, d)) < 0.5 + 2.0 ** -57 / 2.0 ** -53


def test_powers_of_two_are_exact_and_extremes_hold(lib):
    e = np.arange(-1022, 1022)
    d = 2.0 ** e.astype(np.float64)
    assert np.array_equal(_run(lib, d), 2.0 ** (-e.astype(np.float64)))
    assert np.array_equal(_run(lib, -d), -(2.0 ** (-e.astype(np.float64))))
    d = np.array([np.nextafter(2.0, 1.0), 1.5 * 2.0 ** -1022, 1.999 * 2.0 ** 1021, 3.0, 7.0, 1.0 / 3.0])
    _check(d, _run(lib, d))


def test_the_refinement_tolerates_seed_errors(lib):
    rng = np.random.default_rng(10)
    d = rng.uniform(0.001, 10.0, 2000)
    for rel in (2.0 ** -22, -(2.0 ** -22)):
        _check(d, _run(lib, d, seed_rel=rel))


def test_out_of_range_gives_nan(lib):
    got = _run(lib, np.array([0.0, -0.0, 5e-324, np.inf, -np.inf, np.nan, 2.0 ** 1022, -1e308]))
    assert np.all(np.isnan(got))
