"""Host checks of the double-float arithmetic of the ENS_FP32X2 kernels
(csrc/df.cuh) and of their Keller-Miksis and relief-valve right-hand sides
(csrc/km_df.cuh, csrc/valve_df.cuh), built for the CPU with g++ (every
function there is __host__ __device__).

The error bounds are those of the double-word algorithms (Joldes, Muller &
Popescu, ACM TOMS 44(2), 2017) in units of u^2 = 2^-48; the right-hand side
is checked against the float64 oracle (Sec. 4.2 equations) relative to the
magnitude of the terms that cancel in N_KM."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2011_01740_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2011_01740_gb300", "csrc")
U2 = 2.0 ** -48
P = ctypes.POINTER(ctypes.c_double)
P_ = P


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("dfhost") / "df_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", f"-I{CSRC}",
                    os.path.join(HERE, "df_host.cpp"), "-o", out], check=True)
    return ctypes.CDLL(out)


def _p(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(P)


def _prims(lib, a, b):
    out = np.zeros((6, a.size))
    lib.prims(a.size, _p(a), _p(b), out.ctypes.data_as(P))
    return out


def _rel(x, r):
    return np.abs(x - r) / np.abs(r)


def test_double_word_operations_meet_their_error_bounds(lib):
    rng = np.random.default_rng(2)
    n = 100_000
    a = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-10, 10, n)
    b = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-10, 10, n)
    oa, ob = _prims(lib, a, b), _prims(lib, b, a)
    xa, xb = oa[4], ob[4]                       # the pairs as doubles (exact)
    assert _rel(xa, a).max() <= 2.0 * U2        # double -> pair -> double
    assert _rel(oa[1], xa * xb).max() <= 5.0 * U2 + 2.0 ** -52
    # accurate addition: absolute error below 3 u^2 of the operands' magnitude
    assert (np.abs(oa[0] - (xa + xb)) / (np.abs(xa) + np.abs(xb))).max() <= 3.0 * U2 + 2.0 ** -52
    assert np.array_equal(oa[5], _prims(lib, a, -b)[0])          # x - y = x + (-y)
    assert _rel(oa[2], 1.0 / xa).max() <= 4.0 * U2 + 2.0 ** -52
    x = 10.0 ** rng.uniform(-2, 2, n)
    ox = _prims(lib, x, x)
    assert _rel(ox[3], ox[4] ** -0.2).max() <= 4.0 * U2 + 2.0 ** -52


def test_cancellation_is_exact_when_the_result_is_representable(lib):
    # (1 + 2^-30) - 1 = 2^-30 exactly: a float cannot hold 1 + 2^-30, the pair can
    a = np.array([1.0 + 2.0 ** -30, 3.0 + 2.0 ** -40])
    b = np.array([1.0, 3.0])
    out = _prims(lib, a, b)
    assert np.array_equal(out[5], np.array([2.0 ** -30, 2.0 ** -40]))


def test_keller_miksis_right_hand_side_matches_the_oracle(lib):
    rng = np.random.default_rng(1)
    n = 50_000
    phys = dict(pA1=rng.uniform(0, 2e5, n), f1=10 ** rng.uniform(np.log10(2e4), 6, n), pA2=rng.uniform(0, 1e5, n),
                f2=10 ** rng.uniform(np.log10(2e4), 6, n), theta=rng.uniform(0, 6.28, n), RE=np.full(n, 10e-6))
    C = np.ascontiguousarray(oracle.km_coefficients(phys["pA1"], phys["f1"], phys["pA2"], phys["f2"],
                                                    phys["theta"], phys["RE"], oracle.liquid(**W.WATER_25C)))
    t = rng.uniform(0, 1, n)
    y1, y2 = rng.uniform(0.2, 5.0, n), rng.uniform(-3.0, 3.0, n)
    ref = oracle.rhs(oracle.KM, C, t, np.vstack([y1, y2]))[1]
    # the forcing sums of the oracle's equation, handed over as doubles
    w = 2 * np.pi
    fs = C[5] * np.sin(w * t) + C[6] * np.sin(w * C[11] * t + C[12])
    fc = C[7] * np.cos(w * t) + C[8] * np.cos(w * C[11] * t + C[12])
    out = np.zeros(n)
    lib.accel_df(n, _p(C), _p(fs), _p(fc), _p(y1), _p(y2), out.ctypes.data_as(P))
    D = y1 * (1 - C[9] * y2) + C[4] * C[9]
    scale = (np.abs(C[0] + C[1] * y2) * y1 ** -4.2 + np.abs(C[2] * (1 + C[9] * y2)) + np.abs(C[3] + C[4] * y2) / y1
             + np.abs(fs * (1 + C[9] * y2)) + np.abs(y1 * fc) + 1.5 * y2 ** 2) / np.abs(D)
    err = np.abs(out - ref) / scale
    assert np.percentile(err, 99) < 1e-13 and err.max() < 5e-13, (np.percentile(err, 99), err.max())


def test_double_word_square_root(lib):
    """One Newton step on the exact residual of the float square root: within
    4 u^2 of sqrt of the pair's value (measured 3.4 u^2 at most, 1.4 u^2 at
    the 99th percentile); 0 for zero and negative arguments."""
    rng = np.random.default_rng(4)
    x = 10.0 ** rng.uniform(-12, 12, 100_000)
    xs = _prims(lib, x, x)[4]                   # the pairs' exact values
    out = np.zeros_like(x)
    lib.sqrt_df(x.size, _p(x), out.ctypes.data_as(P))
    assert _rel(out, np.sqrt(xs)).max() <= 4.0 * U2
    z = np.array([0.0, -1.0, -1e-30])
    oz = np.ones(3)
    lib.sqrt_df(3, _p(z), oz.ctypes.data_as(P))
    assert np.array_equal(oz, np.zeros(3))


def test_relief_valve_right_hand_side_matches_the_oracle(lib):
    """Eqs. pressure_relief_valve_1-3 in pairs against the float64 oracle on
    random states of the sweep's range (y3 < 0 exercises the clamp), relative
    to the magnitude of the terms that cancel in each component."""
    rng = np.random.default_rng(3)
    n = 50_000
    P = np.vstack([rng.uniform(0.2, 10.0, n), np.full(n, 1.25), np.full(n, 10.0), np.full(n, 20.0), np.full(n, 0.8)])
    y = np.vstack([rng.uniform(-1e-6, 8.0, n), rng.uniform(-20.0, 20.0, n), rng.uniform(-1e-9, 60.0, n)])
    ref = oracle.rhs(oracle.PRV, P, 0.0, y)
    out = np.zeros_like(y)
    lib.valve_df(n, _p(P), _p(y), out.ctypes.data_as(P_))
    scale1 = np.abs(P[1] * y[1]) + np.abs(y[0] + P[2]) + np.abs(y[2])
    scale2 = P[3] * (P[0] + np.abs(y[0]) * np.sqrt(np.maximum(y[2], 0.0)))
    assert np.array_equal(out[0], y[1] + 0.0) or np.abs(out[0] - y[1]).max() <= 2.0 * U2 * np.abs(y[1]).max()
    e1 = np.abs(out[1] - ref[1]) / scale1
    e2 = np.abs(out[2] - ref[2]) / scale2
    assert e1.max() < 2e-14 and e2.max() < 2e-14, (e1.max(), e2.max())


def test_dekker_addition_error_is_bounded_by_the_operands(lib):
    """add_terms (stage sums): |error| <= 2 u^2 (|x| + |y|), also when the sum
    cancels (y near -x)."""
    rng = np.random.default_rng(6)
    n = 100_000
    a = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-6, 6, n)
    b = np.where(rng.uniform(size=n) < 0.5, -a * (1 + rng.uniform(-1e-6, 1e-6, n)),
                 rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-6, 6, n))
    xa, xb = _prims(lib, a, b)[4], _prims(lib, b, a)[4]
    out = np.zeros(n)
    lib.add_terms_df(n, _p(a), _p(b), out.ctypes.data_as(P))
    err = np.abs(out - (xa + xb)) / (np.abs(xa) + np.abs(xb))
    assert err.max() <= 2.0 * U2, err.max() / U2


def test_integer_split_equals_the_subtraction_form_bit_for_bit(lib):
    """from_double takes the low part from the significand bits (integer
    pipe); it must give exactly the pair of the FP64-subtraction form, over
    magnitudes from 2^-120 to 2^120, both signs, exact floats, zero."""
    rng = np.random.default_rng(21)
    x = np.concatenate([rng.choice([-1.0, 1.0], 20000) * 2.0 ** rng.uniform(-120, 120, 20000),
                        rng.uniform(-3.0, 3.0, 5000), [0.0, -0.0, 1.0, -1.5, 2.0 ** -100, 2.0 ** -101,
                                                         np.float32(0.1).astype(np.float64), 1.0 + 2.0 ** -52]])
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(4 * x.size, dtype=np.float32)
    lib.split_df(x.size, x.ctypes.data_as(P), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    o = out.reshape(4, x.size)
    assert np.array_equal(o[0].view(np.uint32), o[2].view(np.uint32))
    assert np.array_equal(o[1].view(np.uint32), o[3].view(np.uint32))
