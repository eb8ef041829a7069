"""Pins of the surrogate-MLP oracle: GELU values, finite-difference gradients,
Adam's first step, and a fit of a known smooth target."""
import math

import numpy as np

from oracle import mlp_oracle as M


def test_gelu_known_values_and_derivative():
    # GELU(z) = z Phi(z): Phi(1) = 0.841344746068543, Phi(-1) = 0.158655253931457
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert abs(M.gelu(np.array([1.0]))[0] - 0.841344746068543) < 1e-15
    assert abs(M.gelu(np.array([-1.0]))[0] + 0.158655253931457) < 1e-15
    assert abs(M.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-16
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - M.gelu_grad(z))) < 1e-9


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    I, H, O = 4, 6, 2
    p = M.init_params(rng, I, H, O)
    for k in p:
        p[k] = p[k] + rng.normal(0, 0.1, p[k].shape)
    X = rng.normal(size=(7, I))
    T = rng.normal(size=(7, O))
    g = M.backward(p, X, T)
    flat = M.flatten(p, I, H, O)
    gflat = M.flatten(g, I, H, O)
    h = 1e-6
    for idx in range(len(flat)):
        e = np.zeros_like(flat)
        e[idx] = h
        lp = M.loss(M.unflatten(flat + e, I, H, O), X, T)
        lm = M.loss(M.unflatten(flat - e, I, H, O), X, T)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[idx]) < 1e-7 * max(1.0, abs(fd)), idx


def test_adam_first_step_moves_each_parameter_by_lr():
    """Bias-corrected Adam: the first update is -lr * g / (|g| + eps)."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=50)
    g = rng.normal(size=50)
    x1, m, v = M.adam_step(x, g, np.zeros(50), np.zeros(50), 1, lr=0.01)
    assert np.max(np.abs((x1 - x) - (-0.01 * g / (np.abs(g) + 1e-8)))) < 1e-15


def test_adam_minimises_a_quadratic():
    x = np.array([3.0, -2.0])
    m = v = np.zeros(2)
    for t in range(1, 3001):
        x, m, v = M.adam_step(x, 2 * x, m, v, t, lr=0.01)
    assert np.max(np.abs(x)) < 1e-2


def test_parameter_count_and_layout():
    assert M.n_params() == 128 * 4 + 128 + 2 * (128 * 128 + 128) + 2 * 128 + 2
    rng = np.random.default_rng(0)
    p = M.init_params(rng)
    assert np.array_equal(M.flatten(M.unflatten(M.flatten(p))), M.flatten(p))
