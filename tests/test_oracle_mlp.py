"""Pins of the surrogate's FP64 oracle (oracle/mlp.py): bf16 rounding,
exact neighbour selection, feature layout, hand-written backward and Adam."""
import numpy as np
import pytest
import torch
from scipy.spatial import cKDTree

from oracle import mlp


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9]])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)
    assert np.array_equal(mlp.bf16(x), want)


def test_knn32_matches_kdtree():
    rng = np.random.default_rng(1)
    mean = rng.uniform(-1, 1, (3000, 3)).astype(np.float32)
    pp = rng.uniform(-1, 1, (50, 3)).astype(np.float32)
    idx = mlp.knn_gaussians(pp, mean)
    q = np.rint(mean.astype(np.float64) * 2 ** 20)
    _, ref = cKDTree(q).query(np.rint(pp.astype(np.float64) * 2 ** 20), k=32)
    assert np.array_equal(idx, ref)


def test_features_layout():
    g = dict(mean=np.array([[0.1, 0.0, 0.0], [0.0, 0.2, 0.0]] + [[5.0, 5.0, 5.0]] * 40, np.float32),
             scale=np.full((42, 3), np.exp(-5.0), np.float32), opacity=np.full(42, 0.5, np.float32),
             rgb=np.tile(np.array([0.1, 0.2, 0.3], np.float32), (42, 1)))
    g["scale"][1] = [np.exp(-4.0), np.exp(-5.0), np.exp(-6.0)]
    pp = np.zeros((1, 3), np.float32)
    f, idx = mlp.probe_features(pp, g)
    assert idx[0, :2].tolist() == [0, 1]
    assert np.allclose(f[0, :10], [1.0, 0, 0, 0, 0, 0, 0.5, 0.1, 0.2, 0.3], atol=1e-6)
    assert np.allclose(f[0, 10:20], [0, 2.0, 0, 1.0, 0, -1.0, 0.5, 0.1, 0.2, 0.3], atol=1e-6)
    # probe at the origin: all sines 0, all cosines 1
    enc = f[0, 320:].reshape(3, 32)
    assert np.allclose(enc[:, :16], 0) and np.allclose(enc[:, 16:], 1)


def _case(seed=2, P=3, B=40):
    rng = np.random.default_rng(seed)
    theta = mlp.init_params(seed)
    theta[mlp.n_params() - 64 - 5 - 320:] += 0.1  # nonzero biases / last layer
    fp = rng.standard_normal((P, mlp.F_PROBE))
    dt = rng.standard_normal((B, 3))
    dt /= np.linalg.norm(dt, axis=1, keepdims=True)
    pidx = rng.integers(0, P, B)
    return rng, theta, fp, dt, pidx


def test_backward_matches_finite_differences():
    """Without operand rounding the network is piecewise linear; central
    differences of <g, y> match the hand-written backward away from ReLU
    kinks (tiny steps, kink crossings detected by two step sizes)."""
    rng, theta, fp, dt, pidx = _case()
    g4 = rng.standard_normal((len(dt), mlp.N_OUT))
    y, a = mlp.forward(theta, fp, dt, pidx, rnd=mlp._ident)
    grad = mlp.backward(a, g4, rnd=mlp._ident)
    f = lambda th: np.sum(g4 * mlp.forward(th, fp, dt, pidx, rnd=mlp._ident)[0])  # noqa: E731
    checked = 0
    for i in rng.choice(mlp.n_params(), 300, replace=False):
        fd = []
        for h in (1e-5, 2.5e-6):
            e = np.zeros_like(theta)
            e[i] = h
            fd.append((f(theta + e) - f(theta - e)) / (2 * h))
        if abs(fd[0] - fd[1]) > 1e-6 * (1 + abs(fd[1])):
            continue  # a ReLU kink within the step
        assert fd[1] == pytest.approx(grad[i], rel=1e-6, abs=1e-8)
        checked += 1
    assert checked > 250


def test_loss_gradient_is_sign_over_count():
    rng, theta, fp, dt, pidx = _case(3)
    target = rng.standard_normal((len(dt), mlp.N_OUT))
    loss, grad, y = mlp.loss_and_grad(theta, fp, dt, pidx, target, rnd=mlp._ident)
    assert loss == pytest.approx(np.abs(y - target).mean())
    _, a = mlp.forward(theta, fp, dt, pidx, rnd=mlp._ident)
    want = mlp.backward(a, np.sign(y - target) / y.size, rnd=mlp._ident)
    assert np.allclose(grad, want, rtol=1e-12, atol=0)


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(4)
    th = rng.standard_normal(100)
    g = rng.standard_normal(100)
    m = v = np.zeros(100)
    t1, m, v = mlp.adam(th, m, v, g, 1, lr=1e-3)
    # first bias-corrected step: lr * g / (|g| + eps)
    assert np.allclose(t1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    t2, m, v = mlp.adam(t1, m, v, g, 2, lr=1e-3)
    assert np.allclose(t2, t1 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_param_count():
    assert mlp.n_params() == 64 * 416 + 64 * 3 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 5 * 64 + 5
