"""Allocation-free entry point (ens_solve_noalloc) against the allocating one.

ens_solve_noalloc serves callers that cannot allocate device memory (memory
owned by another allocator, plugins handed device buffers): it runs the same
kernel on caller-owned buffers with a fixed scratch array in the library.  The
test calls it twice in a row through the C ABI and checks both results against
ens_create / ens_solve / ens_read on the same inputs; the second call checks
that the shared scratch is reset between calls.  This file is collected last.
"""
import numpy as np
import pytest

import paper_2011_01740_gb300 as ens
from paper_2011_01740_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-12   # same kernel and arithmetic: results agree to rounding (in practice bitwise)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _reference(sysid, params, y0, t_span, tol):
    ctx = ens.ens_create(sysid, params.shape[1], params, y0, t_span, ens.ENS_RKCK45, tol)
    try:
        ens.ens_solve(ctx)
        ens.ens_sync(ctx)
        return {k: ens.ens_read(ctx, w) for k, w in (("y", ens.ENS_STATE), ("acc", ens.ENS_ACC),
                                                     ("status", ens.ENS_STATUS), ("nacc", ens.ENS_NSTEPS),
                                                     ("nrej", ens.ENS_NREJ), ("nrhs", ens.ENS_NRHS))}
    finally:
        ens.ens_destroy(ctx)


def _noalloc(sysid, params, y0, t_span, tol, rows, cost_order):
    import torch
    n = params.shape[1]
    dim = y0.shape[0]
    f64 = dict(dtype=torch.float64, device="cuda")
    bufs = dict(y=torch.empty((dim, n), **f64), t=torch.empty(n, **f64), dt=torch.empty(n, **f64),
                acc=torch.empty((rows, n), **f64), status=torch.empty(n, dtype=torch.int32, device="cuda"),
                nacc=torch.empty(n, dtype=torch.int64, device="cuda"),
                nrej=torch.empty(n, dtype=torch.int64, device="cuda"),
                nrhs=torch.empty(n, dtype=torch.int64, device="cuda"))
    ens.ens_solve_noalloc(sysid, n, _dev(params), _dev(y0), t_span, tol, bufs["y"], bufs["t"], bufs["dt"],
                          bufs["acc"], bufs["status"], bufs["nacc"], bufs["nrej"], bufs["nrhs"], cost_order)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in bufs.items()}


def _compare(got, ref):
    np.testing.assert_allclose(got["y"], ref["y"], rtol=REL, atol=0)
    np.testing.assert_allclose(got["acc"], ref["acc"], rtol=REL, atol=0, equal_nan=True)
    for k in ("status", "nacc", "nrej", "nrhs"):
        assert np.array_equal(got[k], ref[k]), k


@pytest.mark.parametrize("cost_order", [1, 0])
def test_noalloc_keller_miksis_matches_allocating_solve_twice(cost_order):
    import torch
    assert torch.cuda.is_available()
    km = W.km(32, 48, n_phases=4)
    ph = km["phys"]
    C = ens.ens_km_coefficients(ph["pA1"], ph["f1"], ph["pA2"], ph["f2"], ph["theta"], ph["RE"], km["liquid"])
    t = km["tol"]
    tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                       n_phases=t.n_phases, phase_len=t.phase_len)
    ref = _reference(ens.ENS_SYS_KELLER_MIKSIS, C, km["y0"], (0.0, 1.0), tol)
    for _ in range(2):
        got = _noalloc(ens.ENS_SYS_KELLER_MIKSIS, C, km["y0"], (0.0, 1.0), tol, 2 * t.n_phases, cost_order)
        _compare(got, ref)


def test_noalloc_relief_valve_matches_allocating_solve_twice():
    wl = W.prv(500, t1=32.0)
    t = wl["tol"]
    tol = ens.make_tol(rtol=t.rtol, atol=t.atol, dt0=t.dt0, dt_min=t.dt_min, dt_max=t.dt_max,
                       event_tol=t.event_tol, acc_t_start=t.acc_t_start)
    ref = _reference(ens.ENS_SYS_RELIEF_VALVE, wl["params"], wl["y0"], (t.t0, t.t1), tol)
    for _ in range(2):
        got = _noalloc(ens.ENS_SYS_RELIEF_VALVE, wl["params"], wl["y0"], (t.t0, t.t1), tol, 35, 1)
        _compare(got, ref)


def test_noalloc_rejects_ensembles_beyond_its_scratch():
    import torch
    n = (1 << 20) + 1
    tol = ens.make_tol(n_phases=1)
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ens.EnsError) as e:
        ens.ens_solve_noalloc(ens.ENS_SYS_KELLER_MIKSIS, n, z, z, (0.0, 1.0), tol, z, z, z, z,
                              torch.zeros(1, dtype=torch.int32, device="cuda"),
                              *[torch.zeros(1, dtype=torch.int64, device="cuda")] * 3)
    assert e.value.status == ens.ENS_EINVAL
    assert "1048576" in str(e.value)


def test_noalloc_refuses_host_buffers_before_launching():
    """Every array must be device memory of the current device (or managed
    memory); a pageable host array is refused with ENS_EINVAL and no kernel
    runs on it."""
    import torch
    n = 4
    tol = ens.make_tol(n_phases=1)
    d = lambda *s, dt=torch.float64: torch.zeros(*s, dtype=dt, device="cuda")
    host_y0 = np.zeros((2, n))
    with pytest.raises(ens.EnsError) as e:
        ens.ens_solve_noalloc(ens.ENS_SYS_KELLER_MIKSIS, n, d(13, n), host_y0, (0.0, 1.0), tol, d(2, n), d(n),
                              d(n), d(2, n), d(n, dt=torch.int32), d(n, dt=torch.int64), d(n, dt=torch.int64),
                              d(n, dt=torch.int64))
    assert e.value.status == ens.ENS_EINVAL
    assert "current device" in str(e.value)
    torch.cuda.synchronize()
