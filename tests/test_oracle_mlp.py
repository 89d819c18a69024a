"""Pins of the surrogate network's FP64 oracle (oracle/mlp.py): bf16
rounding, hand-written backward against finite differences, the L1 loss
gradient and Adam's closed-form first steps."""
import numpy as np
import pytest
import torch

from oracle import mlp


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9]])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)
    assert np.array_equal(mlp.bf16(x), want)


def _case(seed=2, B=40):
    from paper_2510_07729_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    theta = I.surrogate_init(seed).astype(np.float64)
    theta[mlp.n_params() - 5 - 320:] += 0.1  # nonzero output layer and bias
    x = rng.standard_normal((B, mlp.N_IN))
    return rng, theta, x


def test_backward_matches_finite_differences():
    """Without operand rounding the network is piecewise linear; central
    differences of <g, y> match the hand-written backward away from ReLU
    kinks (tiny steps, kink crossings detected by two step sizes)."""
    rng, theta, x = _case()
    g4 = rng.standard_normal((len(x), mlp.N_OUT))
    y, a = mlp.forward(theta, x, rnd=mlp._ident)
    grad = mlp.backward(a, g4, rnd=mlp._ident)
    f = lambda th: np.sum(g4 * mlp.forward(th, x, rnd=mlp._ident)[0])  # noqa: E731
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
    rng, theta, x = _case(3)
    target = rng.standard_normal((len(x), mlp.N_OUT))
    loss, grad, y = mlp.loss_and_grad(theta, x, target, rnd=mlp._ident)
    assert loss == pytest.approx(np.abs(y - target).mean())
    _, a = mlp.forward(theta, x, rnd=mlp._ident)
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
    assert mlp.n_params() == 64 * 18 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 5 * 64 + 5


def test_bf16_network_is_the_rounded_network():
    """With bf16 rounding, the forward pass equals the unrounded network on
    rounded weights and features when the hidden activations are exact in
    bf16 (a one-hot feature and power-of-two weights)."""
    theta = np.zeros(mlp.n_params())
    w = mlp.unflatten(theta.copy())
    w["W1"][:] = 0.0
    w["W1"][0, 0] = 0.5
    w["W2"][1, 0] = 2.0
    w["W3"][2, 1] = 0.25
    w["W4"][0, 2] = 4.0
    th = mlp.flatten(w)
    x = np.zeros((1, mlp.N_IN))
    x[0, 0] = 3.0
    y, _ = mlp.forward(th, x)
    assert y[0, 0] == 3.0 * 0.5 * 2.0 * 0.25 * 4.0 and np.all(y[0, 1:] == 0.0)
