"""Pins of the FP64 MLP oracle (oracle/mlp.py) used to check the learned
tuner's GPU training kernels: a forward pass computed by hand, gradients
against central finite differences of the loss, and Adam's first step against
its closed form.  Each pin is chosen so that a plausible mistake (a dropped
ReLU mask, a transposed weight, a missing bias correction) fails it."""
import numpy as np
import pytest

from oracle import mlp


def _net(D, H, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(mlp.param_count(D, H)) * 0.7


def test_param_layout():
    D, H = 3, 4
    p = np.arange(mlp.param_count(D, H), dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, D, H)
    assert W1.shape == (H, D) and W1[1, 0] == D            # row-major W1[out][in]
    assert b1[0] == H * D
    assert W2[0, 1] == H * D + H + 1
    assert b2[0] == H * D + H + H * H
    assert W3[0] == H * D + 2 * H + H * H
    assert b3 == mlp.param_count(D, H) - 1


def test_forward_by_hand():
    # D = 2, H = 2 with values chosen so one unit of each layer is clipped by ReLU
    W1 = [[1.0, -2.0], [0.5, 0.25]]
    b1 = [0.5, -1.0]
    W2 = [[2.0, 1.0], [-1.0, -3.0]]
    b2 = [0.0, 0.5]
    W3 = [1.5, -4.0]
    b3 = 0.25
    p = np.array(sum(W1, []) + b1 + sum(W2, []) + b2 + W3 + [b3])
    x = np.array([[3.0, 1.0]])
    # layer 1: [3 - 2 + 0.5, 1.5 + 0.25 - 1] = [1.5, 0.75]
    # layer 2: [3 + 0.75, -1.5 - 2.25 + 0.5 -> relu 0] = [3.75, 0]
    # output: 1.5 * 3.75 + 0.25 = 5.875
    Y, H1, H2 = mlp.forward(p, x, 2, 2)
    np.testing.assert_array_equal(H1, [[1.5, 0.75]])
    np.testing.assert_array_equal(H2, [[3.75, 0.0]])
    assert Y[0] == 5.875
    # x = [0, 2]: layer 1 [-3.5, -0.5] -> [0, 0]; layer 2 = relu(b2) = [0, 0.5];
    # output -4 * 0.5 + 0.25
    Y, H1, H2 = mlp.forward(p, np.array([[0.0, 2.0]]), 2, 2)
    np.testing.assert_array_equal(H1, [[0.0, 0.0]])
    np.testing.assert_array_equal(H2, [[0.0, 0.5]])
    assert Y[0] == -1.75


def _fd_grad(p, X, T, D, H, h=1e-6):
    g = np.empty_like(p)
    for k in range(p.size):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        g[k] = (mlp.loss(pp, X, T, D, H) - mlp.loss(pm, X, T, D, H)) / (2 * h)
    return g


@pytest.mark.parametrize("D,H,N,seed", [(3, 5, 7, 0), (8, 6, 20, 1), (2, 4, 1, 2)])
def test_backward_matches_finite_differences(D, H, N, seed):
    rng = np.random.default_rng(100 + seed)
    p = _net(D, H, seed)
    X = rng.standard_normal((N, D))
    T = rng.standard_normal(N)
    g = mlp.backward(p, X, T, D, H)
    gfd = _fd_grad(p, X, T, D, H)
    np.testing.assert_allclose(g, gfd, rtol=1e-6, atol=1e-7)


def test_finite_difference_pin_catches_planted_mistakes():
    """The gradient pin is sharp: two plausible slips, planted in a copy of the
    chain rule here, each move some gradient well past its tolerance."""
    D, H, N = 4, 6, 12
    rng = np.random.default_rng(7)
    p = _net(D, H, 3)
    X = rng.standard_normal((N, D))
    T = rng.standard_normal(N)
    gfd = _fd_grad(p, X, T, D, H)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, D, H)
    Y, H1, H2 = mlp.forward(p, X, D, H)
    dY = 2.0 * (Y - T) / N
    d2 = np.outer(dY, W3) * (H2 > 0)
    for mutant in ("transposed_W2", "no_relu_mask"):
        if mutant == "transposed_W2":
            d1 = (d2 @ W2.T) * (H1 > 0)
        else:
            d1 = d2 @ W2
        dW1 = d1.T @ X
        assert np.max(np.abs(dW1.ravel() - gfd[:H * D])) > 1e-3, mutant


def test_adam_first_step_closed_form():
    # from zero moments the bias-corrected step is lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p0 = np.array([1.0, 2.0, 3.0, 4.0])
    lr, eps = 0.01, 1e-8
    p1, m, v = mlp.adam(p0, g, np.zeros(4), np.zeros(4), 1, lr, eps=eps)
    np.testing.assert_allclose(p1, p0 - lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_steps_are_lr():
    # with a constant gradient the bias-corrected moments equal g and g^2 at
    # every step, so each step moves every parameter by lr * sign(g)
    g = np.array([0.5, -0.25])
    p = np.zeros(2)
    m = np.zeros(2)
    v = np.zeros(2)
    for step in range(1, 6):
        p, m, v = mlp.adam(p, g, m, v, step, 0.1, eps=0.0)
    np.testing.assert_allclose(p, [-0.5, 0.5], rtol=1e-12)


def test_training_with_oracle_fits_a_smooth_target():
    # full-batch Adam on the oracle reduces the loss of a smooth target
    D, H, N = 3, 16, 64
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (N, D))
    T = X[:, 0] * 2 - X[:, 1] ** 2 + 0.5 * X[:, 2]
    p = _net(D, H, 9) * 0.5
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = mlp.loss(p, X, T, D, H)
    for step in range(1, 401):
        p, m, v = mlp.adam(p, mlp.backward(p, X, T, D, H), m, v, step, 1e-2)
    assert mlp.loss(p, X, T, D, H) < 0.05 * l0
