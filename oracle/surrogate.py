"""Learned seed of the Hamiltonian self-consistency loop of Algorithm 1, in float64.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper seeds the SCF loop of every step with the linear extrapolation
H_1 = 2 H_0 - H_-1 (Algorithm 1's extrapolation).  H is linear in the potential, so this is
H[V_pred] with V_pred = 2 V_0 - V_-1.  The learned predictor adds a correction dV = s_out * y
to V_pred, where y is produced by a small 3-D convolutional network from the last three
densities; the SCF loop still decides convergence, so the converged step does not depend on
the network, only the number of passes does.  A network whose parameters are all zero
reproduces the paper's predictor exactly.

Network: four 3 x 3 x 3 cross-correlations with zero padding ("same" size),
3 -> 16 -> 16 -> 16 -> 1 channels, SiLU(z) = z / (1 + e^-z) after the first three layers,
nothing after the last:
    y_l[o](p) = b_l[o] + sum_c sum_{t in {-1,0,1}^3} W_l[o][c][t] x_l[c](p + t),  x = 0 outside.
Input features, a fixed invertible recombination of (rho_t, rho_{t-1}, rho_{t-2}):
    x[0] = rho_t / s_0,   x[1] = (rho_t - rho_{t-1}) / s_1,
    x[2] = (rho_t - 2 rho_{t-1} + rho_{t-2}) / s_2.
Target: (V_{t+dt} - 2 V_t + V_{t-dt}) / s_out  (V = V_H + V_xc after the converged steps).
Loss: mean squared error over the interior points (at least R = 4 points -- the receptive
radius of four 3-point layers -- from every face) of every sample of the batch.
Optimiser: Adam (Kingma & Ba, 2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8.

Parameter vector layout: for l = 0..3, W_l as [cout][cin][kz][ky][kx] (k = tap + 1), then
b_l[cout]; 15,601 numbers in all.

Parity: conv3d is pinned against scipy.ndimage.correlate, the backward pass against central
finite differences of the loss, Adam against its closed form for a constant gradient, the
bfloat16 rounding against hand-worked bit patterns (tests/test_oracle_surrogate.py).
"""
from __future__ import annotations

import numpy as np

CHANNELS = (3, 16, 16, 16, 1)
NLAYERS = 4
RADIUS = 4
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def layer_shapes():
    """[(cout, cin)] of the four layers."""
    return [(CHANNELS[l + 1], CHANNELS[l]) for l in range(NLAYERS)]


def num_params() -> int:
    return sum(co * ci * 27 + co for co, ci in layer_shapes())


def unpack(theta: np.ndarray):
    """Flat parameter vector -> [(W [co, ci, 3, 3, 3], b [co])]."""
    out, k = [], 0
    for co, ci in layer_shapes():
        W = theta[k:k + co * ci * 27].reshape(co, ci, 3, 3, 3)
        k += co * ci * 27
        b = theta[k:k + co]
        k += co
        out.append((W, b))
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def init_params(seed: int, gain: float = 1.0) -> np.ndarray:
    """Seeded He-style initialisation (normal, std = gain * sqrt(2 / (27 cin))), zero biases;
    the last layer starts at zero so the untrained predictor is the paper's."""
    rng = np.random.default_rng(seed)
    layers = []
    for l, (co, ci) in enumerate(layer_shapes()):
        if l == NLAYERS - 1:
            W = np.zeros((co, ci, 3, 3, 3))
        else:
            W = rng.standard_normal((co, ci, 3, 3, 3)) * gain * np.sqrt(2.0 / (27 * ci))
        layers.append((W, np.zeros(co)))
    return pack(layers)


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (8 significant bits) by round-to-nearest-even on the
    IEEE bit pattern, returned as float64.  NaN/inf are not expected here."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _shift(xp: np.ndarray, tz: int, ty: int, tx: int, n):
    """x(p + t) for every p from the zero-padded array xp (pad 1 on each side)."""
    Z, Y, X = n
    return xp[..., 1 + tz:1 + tz + Z, 1 + ty:1 + ty + Y, 1 + tx:1 + tx + X]


TAPS = [(tz, ty, tx) for tz in (-1, 0, 1) for ty in (-1, 0, 1) for tx in (-1, 0, 1)]


def conv3d(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[o] = b[o] + sum_c sum_t W[o, c, t] x[c](p + t); x [cin, Z, Y, X], zero outside."""
    n = x.shape[1:]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    y = np.zeros((W.shape[0],) + n)
    for tz, ty, tx in TAPS:
        xs = _shift(xp, tz, ty, tx, n)
        y += np.einsum("oc,czyx->ozyx", W[:, :, tz + 1, ty + 1, tx + 1], xs)
    return y + b[:, None, None, None]


def forward(theta: np.ndarray, x: np.ndarray, bf16_inputs=()):
    """Network output y [Z, Y, X] for one sample x [3, Z, Y, X]; also the per-layer
    (input, pre-activation) pairs needed by the backward pass.  Layers listed in
    `bf16_inputs` see their input rounded to bfloat16 (the tensor-core inference form)."""
    acts = []
    h = x
    for l, (W, b) in enumerate(unpack(theta)):
        if l in bf16_inputs:
            h = bf16_round(h)
        z = conv3d(h, W, b)
        acts.append((h, z))
        h = silu(z) if l < NLAYERS - 1 else z
    return h[0], acts


def interior_mask(n) -> np.ndarray:
    Z, Y, X = n
    m = np.zeros(n)
    R = RADIUS
    if Z > 2 * R and Y > 2 * R and X > 2 * R:
        m[R:Z - R, R:Y - R, R:X - R] = 1.0
    return m


def loss(theta: np.ndarray, xs, ts) -> float:
    """Mean squared error over the interior points of the batch (xs [B, 3, ...], ts [B, ...])."""
    m = interior_mask(ts[0].shape)
    tot = 0.0
    for x, t in zip(xs, ts):
        y, _ = forward(theta, x)
        tot += float(np.sum(m * (y - t) ** 2))
    return tot / (len(xs) * m.sum())


def gradient(theta: np.ndarray, xs, ts):
    """(loss, d loss / d theta) by the chain rule through the four layers."""
    m = interior_mask(ts[0].shape)
    denom = len(xs) * m.sum()
    layers = unpack(theta)
    grads = [(np.zeros_like(W), np.zeros_like(b)) for W, b in layers]
    tot = 0.0
    for x, t in zip(xs, ts):
        y, acts = forward(theta, x)
        r = m * (y - t)
        tot += float(np.sum(r * (y - t)))
        g = (2.0 / denom) * r[None]                      # d loss / d (layer-4 output)
        for l in range(NLAYERS - 1, -1, -1):
            h, z = acts[l]
            gz = g if l == NLAYERS - 1 else g * silu_grad(z)
            W, _ = layers[l]
            n = h.shape[1:]
            hp = np.pad(h, ((0, 0), (1, 1), (1, 1), (1, 1)))
            dW, db = grads[l]
            for tz, ty, tx in TAPS:
                dW[:, :, tz + 1, ty + 1, tx + 1] += np.einsum(
                    "ozyx,czyx->oc", gz, _shift(hp, tz, ty, tx, n))
            db += gz.sum(axis=(1, 2, 3))
            if l > 0:
                # d/dh[c](q) = sum_o sum_t W[o, c, t] gz[o](q - t)
                gp = np.pad(gz, ((0, 0), (1, 1), (1, 1), (1, 1)))
                gh = np.zeros_like(h)
                for tz, ty, tx in TAPS:
                    gh += np.einsum("oc,ozyx->czyx", W[:, :, tz + 1, ty + 1, tx + 1],
                                    _shift(gp, -tz, -ty, -tx, n))
                g = gh
    return tot / denom, pack(grads)


def adam_step(theta, g, m, v, step: int, lr: float):
    """One Adam update (step counts from 1); returns the new (theta, m, v)."""
    m = BETA1 * m + (1.0 - BETA1) * g
    v = BETA2 * v + (1.0 - BETA2) * g * g
    mh = m / (1.0 - BETA1 ** step)
    vh = v / (1.0 - BETA2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + EPS), m, v


def features(rho_t, rho_tm1, rho_tm2, scales) -> np.ndarray:
    """The three input channels from the last three densities (see the module header)."""
    s0, s1, s2 = scales
    return np.stack([rho_t / s0, (rho_t - rho_tm1) / s1, (rho_t - 2.0 * rho_tm1 + rho_tm2) / s2])


def target(v_tp1, v_t, v_tm1, s_out) -> np.ndarray:
    """Scaled residual of the linear extrapolation 2 V_t - V_{t-dt}."""
    return (v_tp1 - 2.0 * v_t + v_tm1) / s_out
