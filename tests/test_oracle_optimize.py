"""Pins of the FP64 oracle of the SOP texture optimisation step (Sec. 3.1.2,
second step: L = L_pbr + lambda_lam L_lam + lambda_sops L_sops, Adam):
Adam's closed forms and central differences of the total loss."""
import numpy as np
import pytest

from paper_2510_07729_gb300 import inputs as I


@pytest.fixture(scope="module")
def opt():
    from oracle import optimize
    return optimize


def test_adam_constant_gradient_closed_form(opt):
    """With a constant gradient g, Adam's bias-corrected moments are g and
    g^2 at every step, so each step moves the parameter by lr g/(|g| + eps):
    by exactly the learning rate, against the gradient's sign."""
    rng = np.random.default_rng(0)
    p0 = rng.uniform(0.3, 0.7, 64)
    g = rng.choice([-1.0, 1.0], 64) * rng.uniform(1.0, 5.0, 64)
    p, m, v = p0.copy(), np.zeros(64), np.zeros(64)
    lr = 1e-3
    for t in range(1, 51):
        p, m, v = opt.adam(p, g, m, v, t, lr, -np.inf, np.inf)
        step = lr * np.abs(g) / (np.abs(g) + opt.EPS)
        np.testing.assert_allclose(p, p0 - t * step * np.sign(g), rtol=0, atol=1e-13)


def test_adam_clamp_and_zero_gradient(opt):
    p = np.array([0.0, 1.0, 0.5])
    g = np.array([1.0, -1.0, 0.0])
    q, m, v = opt.adam(p, g, np.zeros(3), np.zeros(3), 1, 0.01, 0.0, 1.0)
    assert np.array_equal(q, [0.0, 1.0, 0.5])  # pushed out of range, clamped back; no gradient, no move


def test_l1_loss_gradient(opt):
    rng = np.random.default_rng(1)
    C = rng.uniform(0, 1, (50, 3))
    Ct = rng.uniform(0, 1, (50, 3))
    l, g = opt.l1_loss_grad(C, Ct)
    assert l == pytest.approx(np.abs(C - Ct).mean(), rel=1e-15)
    h = 1e-7
    for idx in [(0, 0), (7, 2), (49, 1)]:
        Cp, Cm = C.copy(), C.copy()
        Cp[idx] += h
        Cm[idx] -= h
        fd = (opt.l1_loss_grad(Cp, Ct)[0] - opt.l1_loss_grad(Cm, Ct)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6)


@pytest.fixture(scope="module")
def problem():
    """A 64-point tiny case: synthetic probe maps as the parameters, another
    draw as the traced targets, a target image from perturbed materials."""
    c = I.make_tiny()
    rng = np.random.default_rng(5)
    M = 64
    pts = {k: np.ascontiguousarray(c[k][:M]) for k in ("x", "n", "wo")}
    maps = I.synthetic_maps(rng, 64, 8)
    traced = I.synthetic_maps(rng, 64, 8)
    params = dict(albedo=c["albedo"][:M].astype(np.float64), rough=np.clip(c["rough"][:M], 0.15, 0.95).astype(np.float64),
                  metal=np.clip(c["metal"][:M], 0.05, 0.95).astype(np.float64), env=c["env"].astype(np.float64),
                  maps_rgb=maps["rgb"].astype(np.float64), maps_occ=maps["occ"].astype(np.float64))
    data = dict(pts, probe_pos=c["probe_pos"], K=4, S=32, target=rng.uniform(0, 1, (M, 3)),
                traced_rgb=traced["rgb"].astype(np.float64), traced_occ=traced["occ"].astype(np.float64))
    return params, data


def _total(opt, st, data):
    return opt.gradients(st, data)[0]["total"]


@pytest.mark.parametrize("block,idx", [("albedo", (3, 1)), ("rough", (10,)), ("metal", (20,)), ("env", (8, 16, 0)),
                                       ("env", (2, 30, 2)), ("maps_rgb", (5, 3, 4, 0)), ("maps_occ", (5, 3, 4))])
def test_total_gradient_central_differences(opt, orc, problem, block, idx):
    """d L / d parameter of the assembled step (adjoint of the shading plus
    the regularisers) against central differences of the total loss. The
    forward reads the parameters in float32, so the step is the float32
    difference of the perturbed values."""
    params, data = problem
    st = opt.init_state(params)
    _, grads = opt.gradients(st, data)
    h = 2e-3 if block == "env" else 1e-3
    p0 = st[block][idx]
    vals = []
    hs = []
    for sgn in (1, -1):
        q = opt.init_state(params)
        q[block][idx] = p0 + sgn * h
        hs.append(float(np.float32(p0 + sgn * h)) - float(np.float32(p0)))
        vals.append(_total(opt, q, data))
    fd = (vals[0] - vals[1]) / (hs[0] - hs[1])
    g = grads[block][idx]
    assert g == pytest.approx(fd, rel=2e-3, abs=1e-7), (block, idx, g, fd)


def test_step_lowers_the_loss(opt, orc, problem):
    params, data = problem
    st = opt.init_state(params)
    losses = [opt.step(st, data)[0]["total"] for _ in range(4)]
    assert losses[-1] < losses[0]
    assert np.all(st["rough"] >= 0.1) and np.all(st["maps_occ"] <= 1.0) and np.all(st["env"] >= 0.0)
