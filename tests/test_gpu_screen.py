"""The surrogate-screened scan end to end on a small grid: the trained
ensemble replaces the FP64 solver on the points it agrees on, the solver
re-solves the rest, and the merged map is checked against a plain FP64 solve
of a validation sample.  Shows what the network gains over the solver alone
(time) and at what error."""
import numpy as np
import pytest

import paper_2011_01740_gb300 as ens
from paper_2011_01740_gb300 import screen

pytestmark = pytest.mark.gpu


def test_screened_scan_small():
    import torch
    assert torch.cuda.is_available()
    r = screen.run(ens, train_shape=(96, 96), screen_m=256, n_phases=16, first_phase=8, threshold=0.05,
                   epochs=80, batch=512, validate=1024)
    print({k: v for k, v in r.items()})
    assert r["train_loss_first_last"][1] < 0.5 * r["train_loss_first_last"][0]
    assert 0.0 < r["fallback_fraction"] < 1.0
    v = r["validation"]
    # re-solved points carry the solver's own value; the rest the surrogate's
    assert v["abs_err_unflagged_p90"] is None or v["abs_err_unflagged_p90"] < 0.25
    assert r["speedup_vs_fp64_estimate"] > 1.0
