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


# ---- forward pass on hand-set weights, worked out unit by unit ----------------------------
# Offsets of the flat parameter vector: W1[128][3] b1 W2[128][128] b2 W3 b3 W4 b4 W5[1][128] b5.
_OFF = {}
_k = 0
for _name, (_o, _i) in zip(("1", "2", "3", "4", "5"), M.SHAPES):
    _OFF["W" + _name], _OFF["b" + _name] = _k, _k + _o * _i
    _k += _o * _i + _o


def _hand_params():
    """A few BF16-exact weights wired asymmetrically (W[out][in]); everything else zero."""
    p = np.zeros(M.N_PARAMS)

    def W(layer, out, inp, val):
        n_in = M.SHAPES[int(layer) - 1][1]
        p[_OFF["W" + layer] + out * n_in + inp] = val

    def b(layer, out, val):
        p[_OFF["b" + layer] + out] = val

    W("1", 0, 0, 1.0), W("1", 1, 1, 2.0), W("1", 2, 2, -0.5), b("1", 0, 0.5), b("1", 3, -1.0)
    W("2", 0, 1, 1.0), W("2", 1, 0, 0.5), W("2", 2, 3, -2.0), W("2", 3, 2, 3.0), b("2", 1, 0.25)
    W("3", 0, 0, 1.0), W("3", 0, 2, 0.5), W("3", 1, 1, 1.0), W("3", 2, 3, -1.0), b("3", 5, 0.75)
    W("4", 0, 0, 2.0), W("4", 1, 5, 1.0), W("4", 2, 1, -1.0), W("4", 3, 2, 1.5), b("4", 0, -0.5)
    W("5", 0, 0, 1.0), W("5", 0, 1, -2.0), W("5", 0, 2, 0.5), W("5", 0, 3, 4.0), b("5", 0, 0.125)
    return p


def _g(z):
    return 0.5 * z * (1.0 + math.erf(z / math.sqrt(2.0)))


def _hand_forward(x0, x1, x2, act=_g, out_act=lambda z: z):
    """The network of _hand_params evaluated unit by unit (only the non-zero units)."""
    h1 = [act(x0 + 0.5), act(2.0 * x1), act(-0.5 * x2), act(-1.0)]
    h2 = [act(h1[1]), act(0.5 * h1[0] + 0.25), act(-2.0 * h1[3]), act(3.0 * h1[2])]
    h3 = {0: act(h2[0] + 0.5 * h2[2]), 1: act(h2[1]), 2: act(-h2[3]), 5: act(0.75)}
    h4 = [act(2.0 * h3[0] - 0.5), act(h3[5]), act(-h3[1]), act(1.5 * h3[2])]
    return out_act(h4[0] - 2.0 * h4[1] + 0.5 * h4[2] + 4.0 * h4[3] + 0.125)


_X = np.array([[1.0, -0.75, 1.5], [0.0, 0.0, 0.0], [-2.0, 1.25, -3.0]])


def test_forward_on_hand_set_weights():
    """oracle.mlp.forward against the unit-by-unit evaluation with math.erf's GELU; the
    weights are BF16-exact, so the BF16 rounding of the reference leaves them unchanged."""
    p = _hand_params()
    assert np.array_equal(M.bf16_round(p), p)
    y, zs = M.forward(p, _X)
    want = np.array([_hand_forward(*r) for r in _X])
    assert np.allclose(y, want, rtol=1e-15, atol=1e-15), (y, want)
    # zero units stay zero (GELU(0) = 0) and the pre-activation of unit 5 of layer 3 is its bias
    assert np.all(zs[0][:, 4:] == 0.0) and np.all(zs[2][:, 5] == 0.75)


def test_forward_pin_catches_wiring_mistakes(monkeypatch):
    """Plant the mistakes the pin must catch in the oracle (on the CPU): weights read as
    W[in][out], GELU dropped from a hidden layer or added on the output, biases shifted."""
    p = _hand_params()
    want = np.array([_hand_forward(*r) for r in _X])

    def far(y):
        return np.max(np.abs(y - want)) > 1e-3

    real_layers = M.layers

    def transposed(params):
        return [(W.reshape(W.shape[::-1]).T if W.shape[0] == W.shape[1] else W, b)
                for W, b in real_layers(params)]

    monkeypatch.setattr(M, "layers", transposed)
    assert far(M.forward(p, _X)[0])
    monkeypatch.setattr(M, "layers", real_layers)

    def shifted_bias(params):
        out = real_layers(params)
        return [(W, np.roll(b, 1)) for W, b in out]

    monkeypatch.setattr(M, "layers", shifted_bias)
    assert far(M.forward(p, _X)[0])
    monkeypatch.setattr(M, "layers", real_layers)
    monkeypatch.setattr(M, "gelu", lambda z: z)
    assert far(M.forward(p, _X)[0])
    monkeypatch.undo()
    # a GELU missing from the hidden layers, or one applied to the output as well
    assert far(np.array([_hand_forward(*r, act=lambda z: z) for r in _X]))
    assert far(np.array([_hand_forward(*r, out_act=_g) for r in _X]))
    assert not far(M.forward(p, _X)[0])
