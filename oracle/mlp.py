"""Learned car-dynamics surrogate, FP64 (test infrastructure only).

The model (not in the paper; the learned-dynamics extension of the car workload):

  features  z = phi(x, u) in R^16: (X, Y, wrap(psi), vx, vy, r, delta) and the two
            controls, each shifted and scaled by fixed constants (psi wrapped to
            (-pi, pi], so the features are 2 pi-periodic in psi), zero padding to 16
  network   h1 = tanh(W1 z + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3
            (W1 256x16, W2 256x256, W3 16x256; outputs 7..15 unused)
  step      x' = x + y[0:7] * out_scale          (a learned state increment)
  loss      L = (1/B) sum_b sum_{i<7} (y_bi - t_bi)^2, t = (x' - x) / out_scale
  optimiser Adam (Kingma and Ba, 2015) with bias correction.

Pins (tests/test_oracle_pins.py): the backward pass against central finite differences,
the first Adam step against its closed form, feature periodicity in psi, and a zero
output layer giving x' = x.
"""
from __future__ import annotations

import math

import numpy as np

from . import systems

IN_CENTER = np.array([0.0, 0.0, 0.0, 5.0, 0.0, 0.0, 0.0])
IN_SCALE = np.array([1 / 20.0, 1 / 20.0, 1 / math.pi, 1 / 5.0, 1 / 2.0, 1 / 3.0, 1 / 0.5])
U_SCALE = np.array([1 / 1.6, 1 / 1.8])
N_IN, N_HID, N_OUT, N_STATE = 16, 256, 16, 7
PARAM_SHAPES = {"W1": (N_HID, N_IN), "b1": (N_HID,), "W2": (N_HID, N_HID), "b2": (N_HID,),
                "W3": (N_OUT, N_HID), "b3": (N_OUT,)}


def wrap_angle(a):
    """Angle in (-pi, pi]."""
    return a - 2.0 * math.pi * np.ceil((a - math.pi) / (2.0 * math.pi))


def features(x, u):
    """x [7][K], u [2][K] -> z [16][K]."""
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    K = x.shape[1]
    z = np.zeros((N_IN, K))
    xs = x.copy()
    xs[2] = wrap_angle(x[2])
    z[:7] = (xs - IN_CENTER[:, None]) * IN_SCALE[:, None]
    z[7:9] = u * U_SCALE[:, None]
    return z


def init_params(seed: int = 0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (input rows 9..15
    and output rows 7..15 of the padded matrices start at zero)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, fan_in, shape in (("W1", 9, (N_HID, N_IN)), ("W2", N_HID, (N_HID, N_HID)), ("W3", N_HID, (N_OUT, N_HID))):
        a = 1.0 / math.sqrt(fan_in)
        p[name] = rng.uniform(-a, a, shape)
    p["W1"][:, 9:] = 0.0
    p["W3"][N_STATE:, :] = 0.0
    p["b1"], p["b2"], p["b3"] = np.zeros(N_HID), np.zeros(N_HID), np.zeros(N_OUT)
    return p


def round_bf16(a):
    """Round to the nearest bfloat16 value (ties to even), returned as float64.  bfloat16
    keeps the sign, the 8 exponent bits and the top 7 fraction bits of a float32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def round_e4m3(a):
    """Round to the nearest E4M3 value (1 sign, 4 exponent bits with bias 7, 3 fraction
    bits; ties to even; largest finite 448, smallest subnormal 2^-9), saturating at 448."""
    a = np.asarray(a, dtype=np.float64)
    s = np.sign(a)
    x = np.minimum(np.abs(a), 448.0)
    e = np.floor(np.log2(np.maximum(x, 2.0 ** -9)))
    e = np.maximum(e, -6.0)                       # below 2^-6 the spacing is fixed (subnormals)
    step = 2.0 ** (e - 3)
    q = np.round(x / step) * step                 # numpy rounds halves to even
    return s * np.minimum(q, 448.0)


def quantize_e4m3_weights(p):
    """Weights as the FP8 kernel sees them: per-tensor scale s = max|W| / 448, W ~ s * e4m3(W / s)."""
    out = {}
    for k, v in p.items():
        v = np.asarray(v, dtype=np.float64)
        if k.startswith("W"):
            m = float(np.abs(np.asarray(v, np.float32)).max())
            s = np.float64(np.float32(m / 448.0)) if m > 0 else 1.0
            out[k] = round_e4m3(np.asarray(v, np.float32).astype(np.float64) / s) * s
        else:
            out[k] = v
    return out


def forward(p, z, act_round=None):
    """z [16][B] -> (y [16][B], cache).  act_round (e.g. round_bf16) is applied to the
    network input and to both hidden activations: the storage precision of a kernel
    that keeps them in that format between its matrix products."""
    q = act_round or (lambda a: a)
    z = q(z)
    h1 = q(np.tanh(p["W1"] @ z + p["b1"][:, None]))
    h2 = q(np.tanh(p["W2"] @ h1 + p["b2"][:, None]))
    y = p["W3"] @ h2 + p["b3"][:, None]
    return y, (z, h1, h2)


def loss_and_grads(p, z, t):
    """MSE over the first 7 outputs, averaged over the batch, and its gradients."""
    y, (z, h1, h2) = forward(p, z)
    B = z.shape[1]
    r = np.zeros_like(y)
    r[:N_STATE] = y[:N_STATE] - t[:N_STATE]
    loss = float((r * r).sum() / B)
    dy = 2.0 * r / B
    g = {"W3": dy @ h2.T, "b3": dy.sum(1)}
    dz2 = (p["W3"].T @ dy) * (1.0 - h2 * h2)
    g["W2"], g["b2"] = dz2 @ h1.T, dz2.sum(1)
    dz1 = (p["W2"].T @ dz2) * (1.0 - h1 * h1)
    g["W1"], g["b1"] = dz1 @ z.T, dz1.sum(1)
    return loss, g


def adam_init(p):
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in p.items()}, "v": {k: np.zeros_like(v) for k, v in p.items()}}


def adam_step(p, g, st, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place: m, v moments with bias correction."""
    st["t"] += 1
    t = st["t"]
    for k in p:
        st["m"][k] = beta1 * st["m"][k] + (1 - beta1) * g[k]
        st["v"][k] = beta2 * st["v"][k] + (1 - beta2) * g[k] * g[k]
        mh = st["m"][k] / (1 - beta1 ** t)
        vh = st["v"][k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def predict(p, out_scale, x, u, act_round=None):
    """x' = x + y[0:7] * out_scale for x [7][K], u [2][K]."""
    y, _ = forward(p, features(x, u), act_round)
    return np.asarray(x, dtype=np.float64) + y[:N_STATE] * np.asarray(out_scale, dtype=np.float64)[:, None]


class CarMLP(systems.Car):
    """The car workload with the learned step in place of the analytic one (same cost).
    act_round=round_bf16 models a network whose inputs and hidden activations are stored
    in bfloat16 (weights are passed already rounded by the caller)."""

    def __init__(self, dt, cost_map, origin, h, params, out_scale, act_round=None, **kw):
        super().__init__(dt, cost_map, origin, h, **kw)
        self.params, self.out_scale = params, np.asarray(out_scale, dtype=np.float64)
        self.act_round = act_round

    def step(self, x, v):
        return predict(self.params, self.out_scale, x, v, self.act_round)
