"""Pins of the oracle's learned predictor (conv3d network, backward pass, Adam, bfloat16)
against results fixed independently of its own code."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import surrogate as sg


def test_conv3d_equals_scipy_correlate():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, 5, 6, 7))
    W = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    y = sg.conv3d(x, W, b)
    for o in range(4):
        ref = b[o] + sum(ndimage.correlate(x[c], W[o, c], mode="constant", cval=0.0)
                         for c in range(3))
        assert np.max(np.abs(y[o] - ref)) < 1e-12


def test_conv3d_is_not_a_flipped_convolution():
    # an asymmetric kernel: correlation, not convolution (the tap t reads x(p + t))
    x = np.zeros((1, 5, 5, 5))
    x[0, 2, 2, 3] = 1.0                     # one point at +1 in x
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 1, 1, 2] = 2.0                  # tap (0, 0, +1)
    y = sg.conv3d(x, W, np.zeros(1))
    assert y[0, 2, 2, 2] == 2.0 and np.count_nonzero(y) == 1


def test_zero_network_is_the_linear_extrapolation():
    theta = np.zeros(sg.num_params())
    rng = np.random.default_rng(1)
    y, _ = sg.forward(theta, rng.standard_normal((3, 9, 9, 9)))
    assert np.all(y == 0.0)
    # the default initialisation also starts at the paper's predictor
    y0, _ = sg.forward(sg.init_params(3), rng.standard_normal((3, 9, 9, 9)))
    assert np.all(y0 == 0.0)
    assert sg.num_params() == 1312 + 6928 + 6928 + 433


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(7)
    n = (10, 9, 11)                          # interior = 2 x 1 x 3 points (R = 4)
    xs = rng.standard_normal((2, 3) + n)
    ts = rng.standard_normal((2,) + n)
    theta = sg.init_params(11, gain=1.5)
    theta[-(16 * 27 + 1):] = 0.3 * rng.standard_normal(16 * 27 + 1)   # non-zero last layer
    L, g = sg.gradient(theta, xs, ts)
    assert abs(L - sg.loss(theta, xs, ts)) < 1e-12 * max(1.0, abs(L))
    # one entry from each layer's W and b plus random ones
    offs, k = [], 0
    for co, ci in sg.layer_shapes():
        offs += [k + 13, k + co * ci * 27 + co - 1]
        k += co * ci * 27 + co
    picks = offs + list(rng.integers(0, sg.num_params(), 8))
    for i in picks:
        h = 1e-5
        tp = theta.copy()
        tp[i] += h
        tm = theta.copy()
        tm[i] -= h
        fd = (sg.loss(tp, xs, ts) - sg.loss(tm, xs, ts)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adam_constant_gradient_closed_form():
    # constant g: m_hat = g and v_hat = g^2 exactly after bias correction, so every step moves
    # each parameter by lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3])
    th = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    lr = 1e-2
    for step in range(1, 6):
        th, m, v = sg.adam_step(th, g, m, v, step, lr)
        assert np.allclose(th, -step * lr * g / (np.abs(g) + sg.EPS), rtol=1e-12, atol=0)


@pytest.mark.parametrize("value,expect", [
    (1.0, 1.0),
    (1.0 + 2.0 ** -7, 1.0 + 2.0 ** -7),          # representable (7 stored bits)
    (1.0 + 2.0 ** -8, 1.0),                       # tie -> even (down)
    (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),       # tie -> even (up)
    (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7),  # above the tie -> up
    (-3.140625, -3.140625),
    (0.1, 0.10009765625),
])
def test_bf16_round(value, expect):
    assert sg.bf16_round(np.array([value]))[0] == expect


def test_features_and_target_recombination():
    rng = np.random.default_rng(2)
    r0, r1, r2 = rng.random((3, 4, 4, 4))
    x = sg.features(r0, r1, r2, (2.0, 0.5, 0.25))
    # the three channels determine the three densities back
    assert np.allclose(x[0] * 2.0, r0)
    assert np.allclose(r0 - x[1] * 0.5, r1)
    assert np.allclose(2 * r1 - r0 + x[2] * 0.25, r2)
    v = rng.random((3, 4, 4, 4))
    t = sg.target(v[0], v[1], v[2], 0.1)
    # V_pred + s_out t reproduces V_{t+dt}
    assert np.allclose(2 * v[1] - v[2] + 0.1 * t, v[0])
