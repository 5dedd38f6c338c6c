"""FP64 CPU reference of the surrogate MLP (6 -> 128 -> 128 -> 128 -> 3, GELU).

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): forward, analytic backward and one
Adam step in plain numpy, written from the definitions, used to check the CUDA
training kernels.  Its own gradient is pinned against central finite differences in
tests/test_oracle_mlp.py.  The parameter layout follows the documented flat layout
(W1 [128][6], b1, W2 [128][128], b2, W3, b3, W4 [3][128], b4).
"""
import math

import numpy as np
from scipy.special import erf

SIZES = ((6, 128), (128, 128), (128, 128), (128, 3))


def unpack(p):
    p = np.asarray(p, np.float64)
    out, off = [], 0
    for fin, fout in SIZES:
        W = p[off:off + fin * fout].reshape(fout, fin)
        off += fin * fout
        b = p[off:off + fout]
        off += fout
        out.append((W, b))
    assert off == p.size
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def forward(p, x):
    """Returns (y, cache) with cache = [(input, pre-activation)] per layer."""
    a = np.asarray(x, np.float64)
    cache = []
    layers = unpack(p)
    for k, (W, b) in enumerate(layers):
        z = a @ W.T + b
        cache.append((a, z))
        a = gelu(z) if k < len(layers) - 1 else z
    return a, cache


def backward(p, cache, dy):
    """Gradient of sum(dy * y) with respect to the flat parameters."""
    layers = unpack(p)
    grads = [None] * len(layers)
    d = np.asarray(dy, np.float64)
    for k in range(len(layers) - 1, -1, -1):
        a, z = cache[k]
        if k < len(layers) - 1:
            d = d * gelu_grad(z)
        W, _ = layers[k]
        grads[k] = (d.T @ a, d.sum(0))
        d = d @ W
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def mse_grad(y, t):
    n = y.size
    return 2.0 * (y - t) / n, float(np.mean((y - t) ** 2))


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
