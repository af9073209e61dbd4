"""Host checks of the integer-pipe sine and cosine of 2 pi x
(csrc/sincos_fx.cuh), built for the CPU with g++ (every function there is
__host__ __device__), against 50-digit arithmetic (mpmath).

The claim under test: the fixed-point evaluation is within 1e-18 of the
exact value before its final rounding, so each result is the correctly
rounded double unless the exact value lies within 1e-18 of a rounding
boundary; exact reduction of x to its fraction of a turn, at any magnitude;
exact values at multiples of 1/4 turn; NaN for NaN and infinite x."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2011_01740_gb300", "csrc")
P = ctypes.POINTER(ctypes.c_double)
SLACK = 1e-18


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("fxhost") / "sincos_fx_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", f"-I{CSRC}",
                    os.path.join(HERE, "sincos_fx_host.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    L.turns_fx.restype = ctypes.c_uint64
    L.turns_fx.argtypes = [ctypes.c_double]
    L.fixed_to_double_fx.restype = ctypes.c_double
    L.fixed_to_double_fx.argtypes = [ctypes.c_uint64]
    return L


def _eval(lib, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    s, c = np.empty_like(x), np.empty_like(x)
    lib.sincos_fx(x.size, x.ctypes.data_as(P), s.ctypes.data_as(P), c.ctypes.data_as(P))
    return s, c


def _exact(x):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    out = []
    for v in x:
        a = 2 * mp.pi * mp.mpf(float(v))        # the double's exact value
        out.append((mp.sin(a), mp.cos(a)))
    return out


def _check(got, exact):
    """|got - exact| within half an ulp of the double nearest exact, plus SLACK."""
    mp = pytest.importorskip("mpmath")
    for g, e in zip(got, exact):
        ulp = float(np.spacing(abs(float(e)))) if e != 0 else 5e-324
        err = float(abs(mp.mpf(float(g)) - e))
        assert err <= 0.5 * ulp + SLACK, (g, e, err, ulp)


def test_random_turns_are_correctly_rounded_within_the_slack(lib):
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.uniform(0.0, 1.0, 3000), rng.uniform(-3.0, 3.0, 1000),
                        rng.uniform(-1e6, 1e6, 500), 10.0 ** rng.uniform(-12, 0, 500)])
    s, c = _eval(lib, x)
    ex = _exact(x)
    _check(s, [e[0] for e in ex])
    _check(c, [e[1] for e in ex])
    # sin^2 + cos^2 = 1 to rounding
    assert np.abs(s * s + c * c - 1.0).max() <= 4.5e-16


def test_quarter_turns_are_exact_and_eighth_turns_correctly_rounded(lib):
    k = np.arange(-16, 17)
    s, c = _eval(lib, k / 4.0)
    ref = {0: (0.0, 1.0), 1: (1.0, 0.0), 2: (0.0, -1.0), 3: (-1.0, 0.0)}
    for kk, ss, cc in zip(k, s, c):
        rs, rc = ref[int(kk) % 4]
        assert ss == rs and cc == rc, (kk, ss, cc)
    x = (2 * np.arange(-8, 8) + 1) / 8.0     # odd eighths: +-sqrt(1/2)
    s, c = _eval(lib, x)
    h = np.sqrt(0.5)
    assert np.all(np.abs(np.abs(s) - h) <= 0.5 * np.spacing(h))
    assert np.all(np.abs(np.abs(c) - h) <= 0.5 * np.spacing(h))
    # the boundaries of the reduction (r = +-1/8 turn) from both sides
    x = np.array([np.nextafter(0.125, 0), np.nextafter(0.125, 1), np.nextafter(0.375, 0), np.nextafter(-0.125, 0)])
    s, c = _eval(lib, x)
    ex = _exact(x)
    _check(s, [e[0] for e in ex])
    _check(c, [e[1] for e in ex])


def test_reduction_is_exact_at_any_magnitude(lib):
    # x = integer + fraction: the integer part drops out exactly
    fr = np.array([0.1, 0.3, 0.7, 0.9375])
    for big in (2.0 ** 20, 2.0 ** 40, 3.0 ** 30):
        x = big + fr
        s, c = _eval(lib, x)
        ex = _exact(x)
        _check(s, [e[0] for e in ex])
        _check(c, [e[1] for e in ex])
    # 2^53 and above are whole numbers of turns
    s, c = _eval(lib, np.array([2.0 ** 53, 2.0 ** 60 + 2.0 ** 8, 1e300, -1e300]))
    assert np.all(s == 0.0) and np.all(c == 1.0)
    # turns() itself: 0.25 -> 2^62, 0.75 -> 3 2^62, -0.25 -> 3 2^62, 2^-64 -> 1
    assert lib.turns_fx(0.25) == 1 << 62 and lib.turns_fx(0.75) == 3 << 62
    assert lib.turns_fx(-0.25) == 3 << 62 and lib.turns_fx(2.0 ** -64) == 1
    assert lib.turns_fx(2.0 ** -65) == 1 and lib.turns_fx(2.0 ** -66) == 0   # ties round up
    assert lib.turns_fx(1.0) == 0 and lib.turns_fx(5e-324) == 0


def test_tiny_arguments_keep_their_absolute_accuracy(lib):
    x = np.array([1e-20, -1e-20, 1e-10, 2.0 ** -40, 0.0, -0.0])
    s, c = _eval(lib, x)
    ex = _exact(x)
    for g, e in zip(s, ex):
        assert abs(float(g) - float(e[0])) <= 1e-18
    assert np.all(c == 1.0)
    assert s[4] == 0.0 and not np.signbit(s[4])


def test_fixed_point_to_double_rounds_to_nearest_even(lib):
    f = lib.fixed_to_double_fx
    assert f(1 << 63) == 0.5 and f(1) == 2.0 ** -64 and f((1 << 64) - 1) == 1.0
    # 2^63 + 2^10 is a tie between 0.5 and 0.5 + 2^-53: even -> 0.5
    assert f((1 << 63) + (1 << 10)) == 0.5
    assert f((1 << 63) + (1 << 10) + 1) == 0.5 + 2.0 ** -53
    assert f((1 << 63) + 3 * (1 << 10)) == 0.5 + 2 * 2.0 ** -53     # tie, odd -> up


def test_nan_and_infinity_give_nan(lib):
    s, c = _eval(lib, np.array([np.nan, np.inf, -np.inf]))
    assert np.all(np.isnan(s)) and np.all(np.isnan(c))
