"""Pins of the oracle's network (learned preconditioner) against finite
differences and against the definition of bfloat16 rounding."""
import numpy as np

from oracle import nn


def test_param_count():
    assert nn.n_params() == 128 * 256 + 256 + 256 * 256 + 256 + 256 * 128 + 128


def test_bf16_rounding():
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e-39])
    r = nn.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -6 and r[3] == -2.5
    assert np.all(np.abs(nn.bf16(np.linspace(-3, 3, 1001)) - np.linspace(-3, 3, 1001)) <= 2.0 ** -8 * 3)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.standard_normal(nn.n_params()) * 0.05
    X = rng.standard_normal((7, 128))
    T = rng.standard_normal((7, 128))
    loss, g = nn.loss_grad(theta, X, T, bf16_store=False)
    idx = rng.choice(nn.n_params(), 40, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (nn.loss_grad(tp, X, T, False)[0] - nn.loss_grad(tm, X, T, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i
