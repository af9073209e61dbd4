"""Host logic of the screening gate (no GPU): the calibration of the
steepness threshold and the disjointness of calibration and validation
samples."""
import numpy as np

from paper_2011_01740_gb300 import screen
from paper_2011_01740_gb300 import workloads as W


def test_gate_calibration_picks_the_largest_threshold_meeting_the_bound():
    """Errors proportional to the steepness, err = 0.1 g with g uniform on
    [0, 1]: the kept points g <= t have p99 error 0.099 t, so the bound 0.05
    is met up to t = 0.505 and not beyond."""
    rng = np.random.default_rng(0)
    g = rng.uniform(0.0, 1.0, 20000)
    err = 0.1 * g
    sd = np.zeros_like(g)
    t = screen.calibrate_gradient_gate(err, sd, g, 0.05, 0.05)
    assert 0.49 < t < 0.51
    assert np.percentile(err[g <= t], 99) <= 0.05
    # points the spread gate already flags do not enter the choice
    sd[g > 0.9] = 1.0
    assert abs(screen.calibrate_gradient_gate(err, sd, g, 0.05, 0.05) - t) < 0.01
    # a bound nothing meets flags every point with a slope
    assert screen.calibrate_gradient_gate(err + 1.0, sd, g, 0.05, 0.05) == 0.0
    # the quantile is a parameter: the median bound is looser
    assert screen.calibrate_gradient_gate(err, np.zeros_like(g), g, 0.05, 0.05, quantile=50.0) > 0.99


def test_calibration_sample_avoids_the_validation_subgrid():
    for m, stride, k in ((256, 2, 4096), (4096, 4, 16384)):
        val = W.screen_subgrid(m, stride)
        cal = W.screen_calibration_points(m, k, stride)
        assert cal.size == k and np.unique(cal).size == k
        assert np.intersect1d(val, cal).size == 0
        assert val.size == ((m + stride - 1) // stride) ** 2
        r, c = cal // m, cal % m
        assert np.all((r % stride != 0) | (c % stride != 0))
