"""FP64 oracle of the learned bake surrogate (test infrastructure only).

The surrogate predicts a probe's octahedral maps (occlusion O, depth D,
radiance RGB) from its local Gaussian neighbourhood and the texel direction,
so that probes can be rebaked quickly after an object moves; the ray-traced
bake remains its fallback and judge.

Model (the reading used throughout; the paper has no surrogate):
  probe features f_p (416): the 32 Gaussians nearest to the probe (exact, by
    the integer squared distance of positions quantised to 2^-20, ties to the
    lower index), nearest first, each as (centre - probe) * 10, log(scale) + 5,
    opacity, rgb (10 values); then a 16-frequency encoding of the probe
    position, sin and cos of pi * 2^(f/3) * p for f = 0..15 and each axis.
  texel input d_t (3): the texel's centre direction (octahedral decode).
  h1 = relu(W1p f_p + W1d d_t + b1)      64
  h2 = relu(W2 h1 + b2)                  64
  h3 = relu(W3 h2 + b3)                  64
  y  = W4 h3 + b4                        5 = (O, D / depth_scale, R, G, B)
Every matrix operand (weights, f_p, d_t, h1, h2, h3, and the back-propagated
deltas fed to the 64x64 layers) is rounded to bfloat16; all sums are exact
here (float64) where the GPU accumulates in float32. Loss: mean absolute
error over the 5 outputs of all samples (an L1 loss, like the L1 texture
supervision of Sec. 3.1.2). Optimiser: Adam (Kingma & Ba 2015), beta1 0.9,
beta2 0.999, eps 1e-8, bias-corrected.
"""
from __future__ import annotations

import numpy as np

NEIGH = 32
N_FREQ = 16
F_PROBE = NEIGH * 10 + 6 * N_FREQ  # 416
HID = 64
N_OUT = 5

# parameter blocks in the flat vector (row-major matrices, out x in)
SHAPES = [("W1p", (HID, F_PROBE)), ("W1d", (HID, 3)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("W4", (N_OUT, HID)), ("b4", (N_OUT,))]
WEIGHTS = ("W1p", "W1d", "W2", "W3", "W4")


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


def _quant(v):
    return np.rint(np.asarray(v, np.float32).astype(np.float64) * 1048576.0).astype(np.int64)


def knn_gaussians(probe_pos, mean, k=NEIGH):
    """Exact k nearest Gaussian centres of each probe (brute force, integer
    keys, ties to the lower index), nearest first."""
    qp, qg = _quant(probe_pos), _quant(mean)
    out = np.empty((len(qp), k), np.int64)
    for i, q in enumerate(qp):
        d = qg - q
        key = (d * d).sum(1).astype(np.uint64)
        order = np.lexsort((np.arange(len(key)), key))
        out[i] = order[:k]
    return out


def probe_features(probe_pos, gauss, idx=None):
    """f_p for every probe [P, 416] (float64, before bf16 rounding)."""
    mean = np.asarray(gauss["mean"], np.float32).astype(np.float64)
    scale = np.asarray(gauss["scale"], np.float32).astype(np.float64)
    op = np.asarray(gauss["opacity"], np.float32).astype(np.float64)
    rgb = np.asarray(gauss["rgb"], np.float32).astype(np.float64)
    pp = np.asarray(probe_pos, np.float32).astype(np.float64)
    if idx is None:
        idx = knn_gaussians(probe_pos, gauss["mean"])
    P = len(pp)
    f = np.empty((P, F_PROBE))
    nb = np.concatenate([(mean[idx] - pp[:, None, :]) * 10.0, np.log(scale[idx]) + 5.0, op[idx][..., None],
                         rgb[idx]], axis=-1)  # [P, 32, 10]
    f[:, :NEIGH * 10] = nb.reshape(P, -1)
    freq = np.pi * 2.0 ** (np.arange(N_FREQ) / 3.0)
    arg = pp[:, :, None] * freq[None, None, :]  # [P, 3, 16]
    enc = np.concatenate([np.sin(arg), np.cos(arg)], axis=-1)  # [P, 3, 32]
    f[:, NEIGH * 10:] = enc.reshape(P, -1)
    return f, idx


def _ident(x):
    return np.asarray(x, np.float64)


def forward(theta, fp, dt, pidx, rnd=bf16):
    """Outputs y [B,5] and the activations for samples (probe pidx[b],
    direction dt[b]). `rnd` is the operand rounding (bf16; identity gives the
    unrounded network, used to pin the derivative formulas)."""
    w = unflatten(theta)
    Wb = {k: rnd(w[k]) for k in WEIGHTS}
    fpb, dtb = rnd(fp), rnd(dt)
    h1p = fpb @ Wb["W1p"].T + w["b1"]
    z1 = h1p[pidx] + dtb @ Wb["W1d"].T
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ Wb["W2"].T + w["b2"]
    h2 = rnd(np.maximum(z2, 0.0))
    z3 = h2 @ Wb["W3"].T + w["b3"]
    h3 = rnd(np.maximum(z3, 0.0))
    y = h3 @ Wb["W4"].T + w["b4"]
    return y, dict(Wb=Wb, fpb=fpb, dtb=dtb, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3, P=len(fp), pidx=pidx)


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
    d1 = (d2 @ Wb["W2"]) * (a["z1"] > 0)
    grads["W1d"] = d1.T @ a["dtb"]
    grads["b1"] = d1.sum(0)
    dh1p = np.zeros((a["P"], HID))
    np.add.at(dh1p, a["pidx"], d1)
    grads["W1p"] = dh1p.T @ a["fpb"]
    return flatten(grads)


def loss_and_grad(theta, fp, dt, pidx, target, rnd=bf16):
    """Mean absolute error over the 5 outputs and its gradient."""
    y, a = forward(theta, fp, dt, pidx, rnd)
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


def init_params(seed):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shp in SHAPES:
        if name.startswith("b"):
            d[name] = np.zeros(shp)
        else:
            fan_in = F_PROBE + 3 if name in ("W1p", "W1d") else shp[1]
            bound = np.sqrt(6.0 / fan_in)
            d[name] = rng.uniform(-bound, bound, shp)
    return flatten(d)
