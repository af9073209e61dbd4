"""Float64 numpy reference of the surrogate network (test infrastructure only).

The surrogate maps the driving of a Keller-Miksis bubble, (log p_A, log f)
scaled to [-1, 1], to two outputs: the log of the maximum expansion ratio and
the logit of "period-1 response".  Network: five affine layers
2 -> 128 -> 128 -> 128 -> 128 -> 2 with the erf form of GELU after the first
four, gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2.  Loss per sample:
squared error on output 0 plus binary cross-entropy with logits on output 1,
averaged over the batch.

Parameter vector of one member (float, this order, W stored [out][in]):
  W1[128][2] b1[128] W2[128][128] b2[128] W3[128][128] b3[128]
  W4[128][128] b4[128] W5[2][128] b5[2]          (50,178 values)

Plain forward and backward passes written from the chain rule; no blocking or
fusion.  Pinned by tests/test_oracle_mlp.py against central finite
differences and closed-form values of the GELU.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

HIDDEN = 128
SHAPES = [("W1", (HIDDEN, 2)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (HIDDEN, HIDDEN)), ("b3", (HIDDEN,)), ("W4", (HIDDEN, HIDDEN)), ("b4", (HIDDEN,)),
          ("W5", (2, HIDDEN)), ("b5", (2,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, off = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = p[off:off + size].reshape(shape)
        off += size
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(p, x):
    """x (n, 2) -> out (n, 2), with the pre-activations of the hidden layers."""
    w = unpack(p)
    h = np.asarray(x, dtype=np.float64)
    zs, hs = [], [h]
    for k in (1, 2, 3, 4):
        z = h @ w[f"W{k}"].T + w[f"b{k}"]
        h = gelu(z)
        zs.append(z)
        hs.append(h)
    out = h @ w["W5"].T + w["b5"]
    return out, (zs, hs)


def loss(out, y):
    """Mean over the batch of (o0 - y0)^2 + BCE-with-logits(o1, y1)."""
    o0, o1 = out[:, 0], out[:, 1]
    mse = (o0 - y[:, 0]) ** 2
    bce = np.maximum(o1, 0.0) - o1 * y[:, 1] + np.log1p(np.exp(-np.abs(o1)))
    return float(np.mean(mse + bce))


def grad(p, x, y):
    """Loss and its gradient with respect to the parameter vector."""
    w = unpack(p)
    out, (zs, hs) = forward(p, x)
    n = out.shape[0]
    L = loss(out, y)
    d_out = np.empty_like(out)
    d_out[:, 0] = 2.0 * (out[:, 0] - y[:, 0]) / n
    d_out[:, 1] = (1.0 / (1.0 + np.exp(-out[:, 1])) - y[:, 1]) / n
    g = {}
    g["W5"] = d_out.T @ hs[4]
    g["b5"] = d_out.sum(axis=0)
    d_h = d_out @ w["W5"]
    for k in (4, 3, 2, 1):
        d_z = d_h * gelu_grad(zs[k - 1])
        g[f"W{k}"] = d_z.T @ hs[k - 1]
        g[f"b{k}"] = d_z.sum(axis=0)
        d_h = d_z @ w[f"W{k}"]
    return L, pack(g)
