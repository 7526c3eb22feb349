"""Pins of the FP64 MLP reference: the gradient against central finite differences, GELU
against its definition, Adam's first step, bf16 rounding on hand-made cases."""
import math

import numpy as np

from oracle import mlp as M


def _params(seed=0, scale=0.2):
    return np.random.default_rng(seed).normal(0.0, scale, size=M.N_PARAMS)


def test_parameter_count():
    assert M.N_PARAMS == 50177


def test_gelu_against_definition_and_derivative():
    for z in (-3.0, -0.7, 0.0, 0.4, 2.5):
        want = 0.5 * z * (1.0 + math.erf(z / math.sqrt(2.0)))
        assert abs(M.gelu(np.array([z]))[0] - want) < 1e-15
        h = 1e-6
        fd = (M.gelu(np.array([z + h]))[0] - M.gelu(np.array([z - h]))[0]) / (2 * h)
        assert abs(M.gelu_grad(np.array([z]))[0] - fd) < 1e-9


def test_gradient_against_central_differences():
    rng = np.random.default_rng(1)
    p = _params(2)
    x = rng.normal(size=(17, 3))
    t = rng.normal(size=17)
    loss, g = M.loss_grad(p, x, t, bf16_weights=False)
    # every layer's weights and biases, including the first and last parameter
    idx = list(rng.choice(M.N_PARAMS, size=60, replace=False)) + [0, 383, 384, 50047, 50048, 50176]
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (M.loss_grad(pp, x, t, False)[0] - M.loss_grad(pm, x, t, False)[0]) / (2 * h)
        assert abs(g[k] - fd) <= 1e-7 + 1e-5 * abs(fd), (k, g[k], fd)
    assert loss > 0


def test_adam_first_step_is_signed_lr():
    """With zero moments, the first bias-corrected step is lr * g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    g = rng.normal(size=100)
    p = rng.normal(size=100)
    lr, eps = 1e-3, 1e-8
    p1, m, v = M.adam(p, np.zeros(100), np.zeros(100), g, lr, 0.9, 0.999, eps, 1)
    assert np.allclose(p - p1, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_cases():
    cases = {1.0: 1.0, 1.0 + 2 ** -8: 1.0, 1.0 + 3 * 2 ** -8: 1.0 + 2 ** -6,
             1.0 + 2 ** -7: 1.0 + 2 ** -7, -2.5: -2.5, 1.0 + 2 ** -8 + 2 ** -20: 1.0 + 2 ** -7}
    for a, b in cases.items():
        assert M.bf16_round(np.array([a]))[0] == b, a
    assert M.bf16_bits(np.array([1.0]))[0] == 0x3F80
