"""FP64 reference of the preconditioner-correction network and its gradient.

ORACLE / TEST INFRASTRUCTURE ONLY.

w(f) = 256^tanh(o), o = w3 . relu(W2 relu(W1 f + b1) + b2) + b3; loss =
mean_i (w(f_i) a_i - b_i)^2.  The weights are rounded to FP16 first (the
network's storage format), as the CUDA forward pass does; the gradient is
with respect to the (unrounded) parameters through that rounding taken as the
identity.  Written out layer by layer with numpy matrix products.
"""
from __future__ import annotations

import numpy as np

IN, W = 8, 64
SHAPES = [(W, IN), (W,), (W, W), (W,), (W,), (1,)]
LOGR = np.log(256.0)


def unpack(p):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(p[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in parts])


def _round_weights(parts):
    w1, b1, w2, b2, w3, b3 = parts
    r = lambda x: x.astype(np.float16).astype(np.float64)
    return r(w1), b1, r(w2), b2, r(w3), b3


def forward(p, f):
    w1, b1, w2, b2, w3, b3 = _round_weights(unpack(p))
    z1 = f @ w1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w2.T + b2
    h2 = np.maximum(z2, 0.0)
    o = h2 @ w3 + b3[0]
    return o, (z1, h1, z2, h2)


def factor(p, f):
    o, _ = forward(p, f)
    return np.exp(LOGR * np.tanh(o))


def loss_grad(p, f, a, b):
    w1, b1, w2, b2, w3, b3 = _round_weights(unpack(p))
    o, (z1, h1, z2, h2) = forward(p, f)
    th = np.tanh(o)
    w = np.exp(LOGR * th)
    err = w * a - b
    n = f.shape[0]
    loss = np.mean(err ** 2)
    do = 2.0 * err * a * w * LOGR * (1.0 - th ** 2) / n
    g_w3 = h2.T @ do
    g_b3 = np.array([do.sum()])
    d2 = np.outer(do, w3) * (z2 > 0)
    g_w2 = d2.T @ h1
    g_b2 = d2.sum(0)
    d1 = (d2 @ w2) * (z1 > 0)
    g_w1 = d1.T @ f
    g_b1 = d1.sum(0)
    return loss, pack([g_w1, g_b1, g_w2, g_b2, g_w3, g_b3])
