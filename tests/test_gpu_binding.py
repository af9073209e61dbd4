"""The Python binding's handling of device tensors handed to asynchronous
C-ABI calls on a side stream."""
import numpy as np
import pytest

import paper_2011_01740_gb300 as ens
from paper_2011_01740_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("pA1", "f1", "pA2", "f2", "theta", "RE")


def test_temporary_device_inputs_outlive_the_queued_kernel():
    """ens_km_coefficients on a side stream with its device inputs created in
    the argument list: their last reference goes when the call returns, while
    the planner kernel may not have run yet.  The binding marks them as used
    by that stream, so the caching allocator does not hand their memory to
    the tensors allocated (and filled on the default stream) right after: the
    coefficients match the host planner's every time."""
    import torch
    km = W.km(512, 512, n_phases=1)
    ph = km["phys"]
    ref = ens.ens_km_coefficients(*[ph[k] for k in KEYS], km["liquid"])      # host planner
    side = torch.cuda.Stream()
    for _ in range(4):
        C = ens.ens_km_coefficients(*[torch.from_numpy(ph[k]).cuda() for k in KEYS], km["liquid"], stream=side)
        junk = [torch.full((ph["pA1"].size,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(12)]
        side.synchronize()
        torch.cuda.synchronize()
        # the device planner equals the host one to an ulp (test_gpu_adaptive);
        # a recycled input would show up as NaN or as another system's values
        np.testing.assert_allclose(C.cpu().numpy(), ref, rtol=4e-16, atol=0)
        del junk
