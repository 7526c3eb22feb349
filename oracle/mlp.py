"""FP64 reference of the MLP surrogate (3 -> 128 -> 128 -> 128 -> 128 -> 1, exact GELU).

TEST INFRASTRUCTURE: only the tests and the benchmark's baseline legs use it.  Weights may
be rounded to BF16 (round to nearest even) first, as the GPU path stores them; everything
after that is float64.  Loss: mean squared error.  Optimiser: Adam with bias correction
(Kingma & Ba, 2015).  Parameter order: W1[128][3] b1 W2[128][128] b2 W3 b3 W4 b4 W5[1][128] b5.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SHAPES = [(128, 3), (128, 128), (128, 128), (128, 128), (1, 128)]
N_PARAMS = sum(o * i + o for o, i in SHAPES)


def bf16_round(a) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a) -> np.ndarray:
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def layers(params):
    """(W, b) views of a flat parameter vector."""
    out, k = [], 0
    for o, i in SHAPES:
        W = params[k:k + o * i].reshape(o, i)
        k += o * i
        b = params[k:k + o]
        k += o
        out.append((W, b))
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, x, bf16_weights: bool = True):
    """y[batch] and the pre-activations of the hidden layers."""
    p = bf16_round(params) if bf16_weights else np.asarray(params, dtype=np.float64)
    h = np.asarray(x, dtype=np.float64)
    zs = []
    L = layers(p)
    for W, b in L[:-1]:
        z = h @ W.T + b
        zs.append(z)
        h = gelu(z)
    W, b = L[-1]
    return (h @ W.T + b)[:, 0], zs


def loss_grad(params, x, target, bf16_weights: bool = True):
    """Mean squared error and its gradient with respect to the (rounded) weights."""
    p = bf16_round(params) if bf16_weights else np.asarray(params, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(target, dtype=np.float64)
    y, zs = forward(p, x, bf16_weights=False)
    B = x.shape[0]
    loss = float(np.mean((y - t) ** 2))
    L = layers(p)
    grads = []
    delta = (2.0 * (y - t) / B)[:, None]  # dL/dy
    hs = [x] + [gelu(z) for z in zs]
    for li in range(len(L) - 1, -1, -1):
        W, b = L[li]
        grads.append((delta.T @ hs[li], delta.sum(0)))
        if li > 0:
            delta = (delta @ W) * gelu_grad(zs[li - 1])
    grads.reverse()
    g = np.concatenate([np.concatenate([gW.ravel(), gb.ravel()]) for gW, gb in grads])
    return loss, g


def adam(p, m, v, g, lr, beta1, beta2, eps, step):
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
