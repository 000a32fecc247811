"""Pins of the proposal-network oracle (oracle/mlp.py) against what the mathematics
fixes: central finite differences of the loss, the composed linear map when every ReLU
passes, the Gaussian log-density of a library routine, Adam's first step, and the BF16
rounding rule."""
import numpy as np
import pytest

from oracle import mlp
from paper_2604_19723_gb300 import workload as W


def _case(B=37, seed=3):
    rng = np.random.default_rng(seed)
    theta = W.mlp_init(seed, out_scale=0.5).astype(np.float64)
    theta[mlp.NPARAM - 16:] = rng.normal(0, 0.1, 16)           # non-zero output biases
    X = rng.normal(size=(B, mlp.IN))
    T = rng.normal(size=(B, mlp.TD))
    return theta, X, T


def test_backward_equals_central_differences():
    theta, X, T = _case()
    g = mlp.backward(theta, X, T)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(mlp.NPARAM, 60, replace=False), np.arange(mlp.NPARAM - 16, mlp.NPARAM)])
    h = 1e-6
    for j in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (mlp.mean_loss(tp, X, T) - mlp.mean_loss(tm, X, T)) / (2 * h)
        assert abs(fd - g[j]) < 1e-6 * max(1.0, abs(fd)), (j, fd, g[j])


def test_forward_is_the_composed_affine_map_when_every_relu_passes():
    rng = np.random.default_rng(1)
    p = {"W1": rng.uniform(0, 1, (64, 16)), "b1": rng.uniform(0, 1, 64), "W2": rng.uniform(0, 1, (64, 64)),
         "b2": rng.uniform(0, 1, 64), "W3": rng.normal(size=(16, 64)), "b3": rng.normal(size=16)}
    theta = mlp.pack(p)
    X = rng.uniform(0, 1, (5, 16))
    y = mlp.forward(theta, X)["y"]
    A = p["W3"] @ p["W2"] @ p["W1"]
    c = p["W3"] @ (p["W2"] @ p["b1"] + p["b2"]) + p["b3"]
    assert np.allclose(y, X @ A.T + c, rtol=1e-12, atol=1e-9)


def test_loss_is_the_gaussian_negative_log_likelihood():
    from scipy.stats import norm
    theta, X, T = _case(B=9)
    y = mlp.forward(theta, X)["y"]
    ref = -np.sum(norm.logpdf(T, loc=y[:, :3], scale=np.exp(y[:, 3:6])), axis=1) - 1.5 * np.log(2 * np.pi)
    assert np.allclose(mlp.loss_terms(y, T), ref, rtol=1e-12, atol=1e-12)


def test_adam_first_step_moves_by_the_learning_rate_against_the_sign():
    g = np.array([3.0, -0.5, 1e-3, -2e-2])
    th, m, v = mlp.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), t=1, lr=0.01, eps=0.0)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_keeps_eight_significant_bits_nearest_even():
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0                      # halfway: to even
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6         # halfway: to even (up)
    assert mlp.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7             # representable
    x = np.random.default_rng(2).normal(size=1000)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= 2 ** -8 * np.abs(x) * (1 + 1e-9))   # half an ulp of 8 bits
