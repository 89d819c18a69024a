"""FP64 oracle of one step of the SOP texture optimisation (test
infrastructure; only the tests may import it).

Sec. 3.1.2, the second reconstruction step: with the shading of the query
(Eq. 2-6), minimise L = L_pbr + lambda_lam L_lam + lambda_sops L_sops over
the environment texels, the per-point albedo, roughness and metallic, and
the SOP textures {L_in, O}, with Adam (Kingma & Ba 2015) at the learning
rates of the implementation details (0.01 for environment and materials,
0.001 for the SOP textures) and weights {lambda_lam, lambda_sops} =
{0.001, 1}.

Readings (the paper is silent or the workload differs):
* L_pbr: the mean absolute error over the shaded points' RGB. The render
  loss adds 0.2 (1 - SSIM) on the image; the shading points of these
  workloads are not an image grid, so that term is left out.
* L_lam = L1(R, 1) + L1(M, 0) and L_sops = L1(L_in, L_tr) + L1(O, O_tr) as
  means over their elements; the traced targets are the ray-traced bake.
* The L1 subgradient at 0 is 0 (sign(0) = 0).
* Adam: beta = 0.9 / 0.999, eps = 1e-8, bias-corrected; after each update a
  parameter is clamped to its range: albedo, metallic and O to [0, 1],
  roughness to [0.1, 1] (the workloads' range; GGX degenerates at 0),
  environment and L_in to [0, inf).
* Gradients of L_pbr come from the query's analytic adjoint (oracle
  query_shade_grad), with the upstream gradient dL/dC.

Parity is pinned by tests/test_oracle_optimize.py: the first Adam step of a
constant-sign gradient moves each parameter by exactly the learning rate,
the L_sops-only loop reaches its closed form, and the loss gradient is
checked against central differences.
"""
from __future__ import annotations

import numpy as np

from . import MODE_SHADE, query_shade, query_shade_grad

LR_MAT = 0.01   # environment, albedo, roughness, metallic
LR_SOP = 0.001  # SOP textures
LAM_LAM = 0.001
LAM_SOPS = 1.0
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8

# parameter block -> (learning rate, clamp low, clamp high)
BLOCKS = {
    "albedo": (LR_MAT, 0.0, 1.0),
    "rough": (LR_MAT, 0.1, 1.0),
    "metal": (LR_MAT, 0.0, 1.0),
    "env": (LR_MAT, 0.0, np.inf),
    "maps_rgb": (LR_SOP, 0.0, np.inf),
    "maps_occ": (LR_SOP, 0.0, 1.0),
}


def l1_loss_grad(C, Ct):
    """Mean absolute error over all elements and its gradient dL/dC."""
    d = np.asarray(C, np.float64) - np.asarray(Ct, np.float64)
    return float(np.abs(d).mean()), np.sign(d) / d.size


def adam(p, g, m, v, t, lr, lo, hi):
    """One bias-corrected Adam step (step number t >= 1), then the clamp."""
    m = BETA1 * m + (1.0 - BETA1) * g
    v = BETA2 * v + (1.0 - BETA2) * g * g
    mh = m / (1.0 - BETA1 ** t)
    vh = v / (1.0 - BETA2 ** t)
    p = np.clip(p - lr * mh / (np.sqrt(vh) + EPS), lo, hi)
    return p, m, v


def init_state(params):
    """FP64 copies of the parameters plus zero Adam moments."""
    st = {"t": 0}
    for k in BLOCKS:
        st[k] = np.array(params[k], np.float64)
        st["m_" + k] = np.zeros_like(st[k])
        st["v_" + k] = np.zeros_like(st[k])
    return st


def gradients(st, data):
    """Loss terms and the gradient of L for every block (no update)."""
    d = data
    C = query_shade(d["x"], d["n"], d["wo"], st["albedo"], st["rough"], st["metal"], d["probe_pos"],
                    st["maps_rgb"], st["maps_occ"], st["env"], d["K"], d["S"], mode=MODE_SHADE)[0]
    l_pbr, gC = l1_loss_grad(C, d["target"])
    g = query_shade_grad(d["x"], d["n"], d["wo"], st["albedo"], st["rough"], st["metal"], d["probe_pos"],
                         st["maps_rgb"], st["maps_occ"], st["env"], d["K"], d["S"], gC)
    M = len(st["rough"])
    l_lam = float(np.abs(st["rough"] - 1.0).mean() + np.abs(st["metal"]).mean())
    l_sops = float(np.abs(st["maps_rgb"] - d["traced_rgb"]).mean() + np.abs(st["maps_occ"] - d["traced_occ"]).mean())
    grads = {
        "albedo": g["albedo"],
        "rough": g["rough"] + LAM_LAM * np.sign(st["rough"] - 1.0) / M,
        "metal": g["metal"] + LAM_LAM * np.sign(st["metal"]) / M,
        "env": g["env"],
        "maps_rgb": g["maps_rgb"] + LAM_SOPS * np.sign(st["maps_rgb"] - d["traced_rgb"]) / st["maps_rgb"].size,
        "maps_occ": g["maps_occ"] + LAM_SOPS * np.sign(st["maps_occ"] - d["traced_occ"]) / st["maps_occ"].size,
    }
    loss = {"pbr": l_pbr, "lam": l_lam, "sops": l_sops, "total": l_pbr + LAM_LAM * l_lam + LAM_SOPS * l_sops}
    return loss, grads


def step(st, data):
    """One optimisation step in place; returns the loss before the update and
    the gradients it used."""
    loss, grads = gradients(st, data)
    st["t"] += 1
    for k, (lr, lo, hi) in BLOCKS.items():
        st[k], st["m_" + k], st["v_" + k] = adam(st[k], grads[k], st["m_" + k], st["v_" + k], st["t"], lr, lo, hi)
    return loss, grads
