"""FP64 oracle of the learned bake surrogate's network (test infrastructure
only).

The surrogate predicts a probe texel's maps (occlusion O, depth D, radiance
RGB) from 18 texel features (oracle.surr_features: the texel direction, the
probe's nearest Gaussians composited along the texel ray, and a coarse
extinction field marched beyond them), so that probes can be rebaked quickly
after an object moves; the ray-traced bake remains its fallback and judge.
The paper has no surrogate (it initialises SOPs by ray tracing, Sec. 3.1.2).

Model (the reading used throughout):
  h1 = relu(W1 x + b1)        x: 18 features, h1: 64
  h2 = relu(W2 h1 + b2)       64
  h3 = relu(W3 h2 + b3)       64
  y  = W4 h3 + b4             5 = (O, D / depth_scale, R, G, B)
Every matrix operand (weights, x, h1, h2, h3, and the back-propagated deltas
of layers 1-3) is rounded to bfloat16; all sums are exact here (float64)
where the GPU accumulates in float32. Loss: mean absolute error over the 5
outputs of all samples (an L1 loss, like the L1 texture supervision of
Sec. 3.1.2). Optimiser: Adam (Kingma & Ba 2015), beta1 0.9, beta2 0.999,
eps 1e-8, bias-corrected.
"""
from __future__ import annotations

import numpy as np

N_IN = 18
HID = 64
N_OUT = 5

# parameter blocks in the flat vector (row-major matrices, out x in)
SHAPES = [("W1", (HID, N_IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, HID)),
          ("b3", (HID,)), ("W4", (N_OUT, HID)), ("b4", (N_OUT,))]
WEIGHTS = ("W1", "W2", "W3", "W4")


def n_params():
    return sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(x):
    """Round to bfloat16 (nearest, ties to even), via float32 as the GPU
    does, returned as float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(x):
    return np.asarray(x, np.float64)


def forward(theta, x, rnd=bf16):
    """Outputs y [B,5] and the activations for features x [B,18]. `rnd` is
    the operand rounding (bf16; identity gives the unrounded network, used
    to pin the derivative formulas)."""
    w = unflatten(theta)
    Wb = {k: rnd(w[k]) for k in WEIGHTS}
    xb = rnd(x)
    z1 = xb @ Wb["W1"].T + w["b1"]
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ Wb["W2"].T + w["b2"]
    h2 = rnd(np.maximum(z2, 0.0))
    z3 = h2 @ Wb["W3"].T + w["b3"]
    h3 = rnd(np.maximum(z3, 0.0))
    y = h3 @ Wb["W4"].T + w["b4"]
    return y, dict(Wb=Wb, xb=xb, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)


def backward(a, g4, rnd=bf16):
    """Gradient w.r.t. theta of sum(g4 * y) given the forward activations."""
    Wb = a["Wb"]
    grads = {"W4": g4.T @ a["h3"], "b4": g4.sum(0)}
    d3 = rnd((g4 @ Wb["W4"]) * (a["z3"] > 0))
    grads["W3"] = d3.T @ a["h2"]
    grads["b3"] = d3.sum(0)
    d2 = rnd((d3 @ Wb["W3"]) * (a["z2"] > 0))
    grads["W2"] = d2.T @ a["h1"]
    grads["b2"] = d2.sum(0)
    d1 = rnd((d2 @ Wb["W2"]) * (a["z1"] > 0))
    grads["W1"] = d1.T @ a["xb"]
    grads["b1"] = d1.sum(0)
    return flatten(grads)


def loss_and_grad(theta, x, target, rnd=bf16):
    """Mean absolute error over the 5 outputs and its gradient."""
    y, a = forward(theta, x, rnd)
    diff = y - target
    g4 = np.sign(diff) / (len(y) * N_OUT)
    return np.abs(diff).mean(), backward(a, g4, rnd), y


def adam(theta, m, v, g, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1). Returns theta, m, v."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
