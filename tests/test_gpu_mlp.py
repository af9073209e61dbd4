"""GPU parity of the surrogate network: BF16 tensor-core forward, backward and
weight gradients against the float64 oracle (oracle/mlp.py), training,
screening and the device helpers of the screening pipeline."""
import numpy as np
import pytest

import paper_2011_01740_gb300 as ens
from oracle import mlp as omlp
from paper_2011_01740_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BF16_TOL = 2e-2      # relative, per output: BF16 operands (8-bit mantissa), FP32 accumulation
# Gradients, element by element: |g - g_ref| <= GRAD_TOL * max |g_ref| within
# each parameter block (the 1e-2 bar for BF16 training), and the block's
# 2-norm within GRAD_TOL as well.  Measured on these batches: at most 7.2e-3
# (element-wise) and 9.2e-3 (norm) over W1..W5 and b1..b4.  The output bias
# b5 (two entries) is the batch sum of the residuals out - y, which have
# mixed signs: the ~0.5 % error of the BF16 forward outputs comes through that
# cancellation amplified (1.3e-2 measured), so b5 takes 2e-2.
GRAD_TOL = 1e-2
GRAD_TOL_B5 = 2e-2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ens.lib()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _model(members, params, train_impl=1):
    m = ens.ens_mlp_create(members, W.SEED)
    ens.ens_mlp_set_params(m, params)
    ens.ens_mlp_set_train_impl(m, train_impl)
    return m


def _loss_grad(p, x, y, impl):
    M, n = p.shape[0], x.shape[0]
    m = _model(M, p, impl)
    try:
        grad = np.empty((M, W.MLP_PARAMS), dtype=np.float32)
        loss = ens.ens_mlp_loss_grad(m, n, _dev(x), _dev(y), M, grad)
        assert ens.ens_mlp_set_train_impl(m, impl) == 0            # no expired tensor-core wait
    finally:
        ens.ens_mlp_destroy(m)
    return loss, grad


def _blocks():
    offs = np.cumsum([0] + [s for s, _ in W.MLP_FAN_IN])
    names = [n for n, _ in omlp.SHAPES]
    return list(zip(names, offs[:-1], offs[1:]))


def test_parameter_layout_matches():
    assert ens.ens_mlp_param_count() == omlp.N_PARAMS == W.MLP_PARAMS


def test_params_round_trip():
    import torch
    p = W.mlp_params(3)
    m = _model(3, p)
    try:
        back = np.empty_like(p)
        ens.ens_mlp_get_params(m, back)
        assert np.array_equal(back, p)
    finally:
        ens.ens_mlp_destroy(m)


@pytest.mark.parametrize("impl", [1, 0])
@pytest.mark.parametrize("n", [1, 77, 128, 1000])
def test_forward_matches_oracle(n, impl):
    """Training-form forward (impl 1: tcgen05, 0: mma.sync)."""
    import torch
    M = 4
    p = W.mlp_params(M)
    x, _ = W.mlp_batch(n)
    m = _model(M, p, impl)
    try:
        out = torch.empty((M, n, 2), dtype=torch.float32, device="cuda")
        ens.ens_mlp_forward(m, n, _dev(x), out)
        torch.cuda.synchronize()
        g = out.cpu().numpy()
    finally:
        ens.ens_mlp_destroy(m)
    for k in range(M):
        ref, _ = omlp.forward(p[k].astype(np.float64), x.astype(np.float64))
        err = np.abs(g[k] - ref).max() / np.abs(ref).max()
        assert err < BF16_TOL, (k, err)


@pytest.mark.parametrize("impl", [1, 0])
@pytest.mark.parametrize("n", [300, 5000])
def test_gradient_matches_oracle(n, impl):
    """Loss and gradient of one batch for every member and every parameter
    block: 300 samples (3 tiles with a ragged tail, 3 weight-gradient slices)
    and 5,000 (8 slices of 640 samples, 5 chunks each, the last one ragged)."""
    M = 4
    p = W.mlp_params(M)
    x, y = W.mlp_batch(n)
    loss, grad = _loss_grad(p, x, y, impl)
    for k in range(M):
        L, g = omlp.grad(p[k].astype(np.float64), x.astype(np.float64), y.astype(np.float64))
        assert abs(loss[k] - L) < 1e-3 * abs(L), (k, loss[k], L)
        for name, lo, hi in _blocks():
            ref = g[lo:hi]
            tol = GRAD_TOL_B5 if name == "b5" else GRAD_TOL
            scale = max(np.abs(ref).max(), 1e-30)
            elem = np.abs(grad[k, lo:hi] - ref) / scale
            assert elem.max() <= tol, (k, name, elem.max(), int(elem.argmax()))
            norm = np.linalg.norm(grad[k, lo:hi] - ref) / max(np.linalg.norm(ref), 1e-30)
            assert norm <= tol, (k, name, norm)


@pytest.mark.parametrize("impl", [1, 0])
def test_screen_agrees_with_member_outputs(impl):
    """Screening (impl 1: tcgen05 kernel with TMEM accumulators, 0: fused
    mma.sync kernel) against the per-member forward outputs and against the
    float64 oracle."""
    import torch
    M, n = 4, 5000
    p = W.mlp_params(M)
    x, _ = W.mlp_batch(n, seed=7)
    m = _model(M, p)
    try:
        ens.ens_mlp_set_screen_impl(m, impl)
        xd = _dev(x)
        out = torch.empty((M, n, 2), dtype=torch.float32, device="cuda")
        ens.ens_mlp_forward(m, n, xd, out)
        mean, sd, p1 = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
        ens.ens_mlp_screen(m, n, xd, mean, sd, p1)
        torch.cuda.synchronize()
        assert ens.ens_mlp_set_screen_impl(m, impl) == 0          # no expired tensor-core wait
    finally:
        ens.ens_mlp_destroy(m)
    o = out.cpu().numpy().astype(np.float64)
    exact = dict(rtol=1e-5, atol=1e-6) if impl == 0 else dict(rtol=2e-2, atol=2e-2)
    np.testing.assert_allclose(mean.cpu().numpy(), o[:, :, 0].mean(0), **exact)
    np.testing.assert_allclose(sd.cpu().numpy(), o[:, :, 0].std(0), rtol=1e-4 if impl == 0 else 5e-2,
                               atol=1e-5 if impl == 0 else 2e-2)
    np.testing.assert_allclose(p1.cpu().numpy(), (1 / (1 + np.exp(-o[:, :, 1]))).mean(0), **exact)
    refs = np.stack([omlp.forward(p[k].astype(np.float64), x.astype(np.float64))[0] for k in range(M)])
    ref_mean = refs[:, :, 0].mean(0)
    err = np.abs(mean.cpu().numpy() - ref_mean).max() / np.abs(ref_mean).max()
    assert err < BF16_TOL, err


def test_screen_tcgen05_large_grid_matches_mma_sync():
    """Many tiles per CTA (persistent walk) and a ragged last tile."""
    import torch
    M, n = 4, 300_001
    p = W.mlp_params(M, seed=5)
    x, _ = W.mlp_batch(n, seed=9)
    m = _model(M, p)
    try:
        xd = _dev(x)
        res = {}
        for impl in (1, 0):
            ens.ens_mlp_set_screen_impl(m, impl)
            outs = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
            ens.ens_mlp_screen(m, n, xd, *outs)
            torch.cuda.synchronize()
            res[impl] = [o.cpu().numpy() for o in outs]
        assert ens.ens_mlp_set_screen_impl(m, 1) == 0
    finally:
        ens.ens_mlp_destroy(m)
    for a, b in zip(res[1], res[0]):
        np.testing.assert_allclose(a, b, rtol=2e-2, atol=2e-2)


def test_tcgen05_gradient_agrees_with_mma_sync():
    """The two training implementations round the same operands to BF16 and
    accumulate in FP32; they differ only in the order of the FP32 sums, so
    their gradients agree far inside the tolerance against the oracle."""
    M, n = 3, 2000
    p = W.mlp_params(M, seed=6)
    x, y = W.mlp_batch(n, seed=8)
    l1, g1 = _loss_grad(p, x, y, 1)
    l0, g0 = _loss_grad(p, x, y, 0)
    np.testing.assert_allclose(l1, l0, rtol=1e-5)
    for k in range(M):
        for name, lo, hi in _blocks():
            err = np.linalg.norm(g1[k, lo:hi] - g0[k, lo:hi]) / max(np.linalg.norm(g0[k, lo:hi]), 1e-30)
            assert err < 2e-3, (k, name, err)


@pytest.mark.parametrize("impl", [1, 0])
def test_training_reduces_loss(impl):
    M, n = 4, 8192
    x, y = W.mlp_batch(n, seed=11)
    m = ens.ens_mlp_create(M, W.SEED)
    ens.ens_mlp_set_train_impl(m, impl)
    try:
        hist = ens.ens_mlp_train(m, n, _dev(x), _dev(y), ens.make_train_cfg(epochs=40, batch=512, lr=2e-3), M)
        assert ens.ens_mlp_set_train_impl(m, impl) == 0
    finally:
        ens.ens_mlp_destroy(m)
    assert hist.shape == (40, M)
    assert np.all(np.isfinite(hist))
    assert np.all(hist[-1] < 0.25 * hist[0]), hist[[0, -1]]


def test_select_gather_scatter_labels_features():
    import torch
    rng = np.random.default_rng(4)
    n = 100_003
    v = rng.uniform(0, 1, n).astype(np.float32)
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    k = ens.ens_select_above(n, _dev(v), 0.9, idx)
    ref = np.nonzero(v > 0.9)[0]
    assert k == ref.size and np.array_equal(idx[:k].cpu().numpy(), ref)
    src = rng.normal(size=n)
    dst = torch.empty(k, dtype=torch.float64, device="cuda")
    ens.ens_gather_f64(k, idx, _dev(src), dst)
    assert np.array_equal(dst.cpu().numpy(), src[ref])
    ys = torch.from_numpy(np.stack([np.arange(k), np.zeros(k)], 1).astype(np.float32)).cuda()
    tgt = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    ens.ens_scatter_labels(k, idx, ys, tgt)
    t = tgt.cpu().numpy()
    assert np.array_equal(t[ref], np.arange(k, dtype=np.float32)) and np.all(t[v <= 0.9] == -1.0)
    # features and labels
    pA, f = W.screen_grid(64)
    x = torch.empty((pA.size, 2), dtype=torch.float32, device="cuda")
    ens.ens_km_features(pA.size, _dev(pA), _dev(f), W.KM_FEATURE_RANGE, x)
    lo_a, hi_a, lo_f, hi_f = W.KM_FEATURE_RANGE
    ex = np.stack([2 * np.log(pA / lo_a) / np.log(hi_a / lo_a) - 1, 2 * np.log(f / lo_f) / np.log(hi_f / lo_f) - 1], 1)
    np.testing.assert_allclose(x.cpu().numpy(), ex, atol=2e-7)
    acc = np.abs(rng.normal(size=(8, 50))) + 1.0
    acc[4::2, :25] = acc[4, :25]           # maxima equal over phases 2, 3: period 1
    y = torch.empty((50, 2), dtype=torch.float32, device="cuda")
    ens.ens_km_labels(50, _dev(acc), 4, 2, 1e-4, y)
    yy = y.cpu().numpy()
    np.testing.assert_allclose(yy[:, 0], np.log(acc[4::2].max(0)), rtol=1e-6)
    assert np.array_equal(yy[:, 1], (np.ptp(acc[4::2], 0) / acc[4::2].max(0) < 1e-4).astype(np.float32))
