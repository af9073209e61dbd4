"""The surrogate-screened scan end to end on a small grid.

The trained ensemble replaces the FP64 solver where both gates pass it (the
configured spread gate, and a steepness gate calibrated on held-out solved
points), the solver re-solves the rest, and the merged map is checked against
a plain FP64 solve of a validation sub-grid that the calibration never saw.
Shows what the network gains over the solver alone (time) and at what error."""
import numpy as np
import pytest

import paper_2011_01740_gb300 as ens
from paper_2011_01740_gb300 import screen
from paper_2011_01740_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# The small case (96 x 96 training grid, 80 epochs) gives a coarser network
# than the benchmark's (362 x 362, 150 epochs; bound p99 <= 0.05 there), so
# its gate is calibrated for the 90th percentile of |ln r error| within 0.08.
QUANTILE, BOUND = 90.0, 0.08


def test_screened_scan_small():
    import torch
    assert torch.cuda.is_available()
    r = screen.run(ens, train_shape=(96, 96), screen_m=256, n_phases=16, first_phase=8, threshold=0.05,
                   bound=BOUND, quantile=QUANTILE, calib_points=4096, val_stride=2, epochs=80, batch=512, lr=2e-3)
    print({k: v for k, v in r.items()})
    assert r["train_loss_first_last"][1] < 0.5 * r["train_loss_first_last"][0]
    assert 0.0 < r["fallback_fraction"] < 1.0
    c = r["calibration"]
    assert c["kept_fraction"] > 0.3 and c["unflagged_err_quantile"] <= BOUND
    v = r["validation"]
    assert v["status"] == ens.ENS_OK
    # the solver's own value replaces the surrogate's at flagged points
    assert v["err_flagged_max"] == 0.0
    # the bound holds out of sample, on the validation sub-grid the
    # calibration never saw, within the sampling error of 4096 points
    unflagged = v["points"] - v["flagged"]
    assert unflagged > 0.3 * v["points"]
    assert v["err_unflagged"]["p90"] <= 1.25 * BOUND
    assert v["period1_error_rate_unflagged"] < 0.1
    assert r["speedup"] > 1.0
    assert set(W.screen_subgrid(256, 2)).isdisjoint(set(W.screen_calibration_points(256, 4096, 2)))
