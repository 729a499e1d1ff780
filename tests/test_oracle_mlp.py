"""Pins of the FP64 network reference: its analytic gradient against central
finite differences (with the weight rounding switched off so the loss is
smooth), and the factor's range [1/256, 256]."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences(monkeypatch):
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.3, mlp.pack([np.zeros(s) for s in mlp.SHAPES]).size)
    f = rng.normal(0, 1, (40, mlp.IN))
    a = rng.normal(0, 1, 40)
    b = rng.normal(0, 1, 40)
    monkeypatch.setattr(mlp, "_round_weights", lambda parts: tuple(parts))
    loss, g = mlp.loss_grad(p, f, a, b)
    idx = rng.choice(p.size, 60, replace=False)
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p); e[i] = eps
        num = (mlp.loss_grad(p + e, f, a, b)[0] - mlp.loss_grad(p - e, f, a, b)[0]) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_factor_range():
    rng = np.random.default_rng(1)
    p = rng.normal(0, 3.0, mlp.pack([np.zeros(s) for s in mlp.SHAPES]).size)
    w = mlp.factor(p, rng.normal(0, 5, (200, mlp.IN)))
    assert np.all(w >= 1 / 256 - 1e-12) and np.all(w <= 256.0 + 1e-12)
    assert w.min() < 0.25 and w.max() > 4.0
