"""Oracle of the proposal network of the learned MT proposal (no counterpart in the paper).

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and the CPU legs of
bench.py; the product path never calls it.

The network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with x in R^16, hidden widths 64,
y in R^16; y[0:3] is the mean and y[3:6] the log standard deviation of a Gaussian over
a 3-vector.  The loss of a batch of B rows is the mean negative log-likelihood of the
targets t (B x 3) without the constant, L = (1/B) sum_i sum_a [(t_ia - y_ia)^2
exp(-2 y_i,3+a) / 2 + y_i,3+a].  Gradients by the chain rule written out layer by layer;
Adam (Kingma and Ba, Algorithm 1) with bias-corrected moments.

FP64 throughout.  With bf16=True the values the GPU stores in BF16 are rounded to BF16
(round to nearest even) at the same places: inputs, weights, the two hidden
activations, and the output and hidden gradients where they enter the weight and data
products (the bias gradients use them unrounded); sums stay FP64.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT, TD = 16, 64, 16, 3
SHAPES = (("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (OUT, H)), ("b3", (OUT,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(x) -> np.ndarray:
    """Round to BF16 (the top 16 bits of the FP32 value, nearest even) and back."""
    b = np.asarray(x, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def forward(theta: np.ndarray, X: np.ndarray, bf: bool = False) -> dict:
    p = unpack(theta)
    q = (lambda a: bf16(a)) if bf else (lambda a: np.asarray(a, np.float64))
    x = q(X)
    z1 = x @ q(p["W1"]).T + p["b1"]
    a1 = q(np.maximum(z1, 0.0))
    z2 = a1 @ q(p["W2"]).T + p["b2"]
    a2 = q(np.maximum(z2, 0.0))
    y = a2 @ q(p["W3"]).T + p["b3"]
    return dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2, y=y)


def loss_terms(y: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Per-row negative log-likelihood without the constant (3/2) log(2 pi)."""
    mu, ls = y[:, :TD], y[:, TD:2 * TD]
    return np.sum(0.5 * (T - mu) ** 2 * np.exp(-2.0 * ls) + ls, axis=1)


def mean_loss(theta, X, T, bf: bool = False) -> float:
    return float(np.mean(loss_terms(forward(theta, X, bf)["y"], T)))


def backward(theta: np.ndarray, X: np.ndarray, T: np.ndarray, bf: bool = False) -> np.ndarray:
    """Gradient of the mean loss with respect to every parameter (packed like theta)."""
    p = unpack(theta)
    c = forward(theta, X, bf)
    q = (lambda a: bf16(a)) if bf else (lambda a: a)
    B = X.shape[0]
    y = c["y"]
    mu, ls = y[:, :TD], y[:, TD:2 * TD]
    e = np.exp(-2.0 * ls)
    d = T - mu
    dy = np.zeros_like(y)
    dy[:, :TD] = -d * e / B
    dy[:, TD:2 * TD] = (1.0 - d * d * e) / B
    g = {"b3": dy.sum(0), "W3": q(dy).T @ c["a2"]}
    da2 = q(dy) @ q(p["W3"])
    dz2 = da2 * (c["z2"] > 0)
    g["b2"] = dz2.sum(0)
    g["W2"] = q(dz2).T @ c["a1"]
    da1 = q(dz2) @ q(p["W2"])
    dz1 = da1 * (c["z1"] > 0)
    g["b1"] = dz1.sum(0)
    g["W1"] = q(dz1).T @ c["x"]
    return pack(g)


def adam(theta, grad, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step; returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
