"""FP64 reference of the surrogate MLP (forward, backward, Adam).

TEST INFRASTRUCTURE ONLY (same rules as oracle.py: only tests/, smoke() and
bench.py's CPU legs may use it; it shares no code with the CUDA kernels).

Network (one ensemble member): x (4) -> 128 -> 128 -> 128 -> y (2), GELU
after each hidden layer, GELU(z) = z * Phi(z) with Phi the standard normal
CDF (the exact form, via erf).  Loss: mean squared error over the batch and
the outputs, L = 1/(B*O) * sum (y - t)^2.  Adam with bias correction.

Flat parameter layout of one member (float order used by the CUDA library):
  W1 [H][I], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H], W4 [O][H], b4 [O]
(row-major, output index first).
"""
import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def shapes(I=4, H=128, O=2):
    return [("W1", (H, I)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
            ("W4", (O, H)), ("b4", (O,))]


def n_params(I=4, H=128, O=2):
    return sum(int(np.prod(s)) for _, s in shapes(I, H, O))


def unflatten(flat, I=4, H=128, O=2):
    out, o = {}, 0
    for name, s in shapes(I, H, O):
        n = int(np.prod(s))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(s)
        o += n
    return out


def flatten(p, I=4, H=128, O=2):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in shapes(I, H, O)])


def forward(p, X):
    """Returns the output and the cache of pre-activations / activations."""
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    A1 = gelu(Z1)
    Z2 = A1 @ p["W2"].T + p["b2"]
    A2 = gelu(Z2)
    Z3 = A2 @ p["W3"].T + p["b3"]
    A3 = gelu(Z3)
    Y = A3 @ p["W4"].T + p["b4"]
    return Y, (X, Z1, A1, Z2, A2, Z3, A3)


def loss(p, X, T):
    Y, _ = forward(p, X)
    return float(np.mean((Y - np.asarray(T, dtype=np.float64)) ** 2))


def backward(p, X, T):
    """Gradient of the MSE loss with respect to every parameter (chain rule)."""
    Y, (X, Z1, A1, Z2, A2, Z3, A3) = forward(p, X)
    B, O = Y.shape
    dY = 2.0 * (Y - np.asarray(T, dtype=np.float64)) / (B * O)
    g = {}
    g["W4"] = dY.T @ A3
    g["b4"] = dY.sum(axis=0)
    dZ3 = (dY @ p["W4"]) * gelu_grad(Z3)
    g["W3"] = dZ3.T @ A2
    g["b3"] = dZ3.sum(axis=0)
    dZ2 = (dZ3 @ p["W3"]) * gelu_grad(Z2)
    g["W2"] = dZ2.T @ A1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * gelu_grad(Z1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return g


def adam_step(flat, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(rng, I=4, H=128, O=2):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    p = {}
    for name, s in shapes(I, H, O):
        if name.startswith("W"):
            bound = 1.0 / math.sqrt(s[1])
            p[name] = rng.uniform(-bound, bound, size=s)
        else:
            p[name] = np.zeros(s)
    return p
