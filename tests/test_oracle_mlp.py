"""Pins of the oracle's network: gradients against finite differences, Adam
against its closed form on a quadratic, and training reducing the loss."""
import numpy as np
import pytest

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params([5, 7, 6, 3], 1)
    for i in range(1, len(p), 2):
        p[i] = rng.standard_normal(p[i].shape) * 0.1     # nonzero biases
    x = rng.standard_normal((9, 5))
    t = rng.standard_normal((9, 3))
    _, g = mlp.loss_and_grad(p, x, t)
    h = 1e-6
    for i in range(len(p)):
        flat = p[i].ravel()
        for j in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[j]
            flat[j] = old + h
            lp, _ = mlp.loss_and_grad(p, x, t)
            flat[j] = old - h
            lm, _ = mlp.loss_and_grad(p, x, t)
            flat[j] = old
            assert g[i].ravel()[j] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)


def test_linear_network_equals_least_squares_gradient():
    # one layer: y = x W + b; dL/dW = 2/(B n) x^T (xW + b - t)
    rng = np.random.default_rng(3)
    W = rng.standard_normal((4, 2))
    b = rng.standard_normal(2)
    x = rng.standard_normal((8, 4))
    t = rng.standard_normal((8, 2))
    loss, g = mlp.loss_and_grad([W, b], x, t)
    r = x @ W + b - t
    assert loss == pytest.approx(np.mean(r ** 2))
    assert np.allclose(g[0], 2.0 / 16 * x.T @ r)
    assert np.allclose(g[1], 2.0 / 16 * r.sum(0))


def test_adam_first_step_is_sign_times_lr():
    # with bias correction the first Adam step is lr * g / (|g| + eps)
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    mlp.adam_step(p, g, m, v, 1, 0.01)
    assert np.allclose(p[0], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01 * 1e-3 / (1e-3 + 1e-8)])


def test_training_fits_a_smooth_map():
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, size=(256, 4))
    t = np.stack([np.sin(x[:, 0]) + x[:, 1] ** 2, x[:, 2] * x[:, 3]], 1)
    p = mlp.init_params([4, 32, 32, 2], 2)
    m = [np.zeros_like(q) for q in p]
    v = [np.zeros_like(q) for q in p]
    l0, _ = mlp.loss_and_grad(p, x, t)
    for step in range(1, 601):
        _, g = mlp.loss_and_grad(p, x, t)
        mlp.adam_step(p, g, m, v, step, 3e-3)
    l1, _ = mlp.loss_and_grad(p, x, t)
    assert l1 < 0.05 * l0


def test_round_bf16_ties_to_even_and_bounds_the_error():
    # spacing of bfloat16 at 1 is 2^-7
    assert mlp.round_bf16(1.0) == 1.0
    assert mlp.round_bf16(1.0 + 2.0 ** -8) == 1.0                       # tie -> even mantissa
    assert mlp.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6        # tie -> even mantissa
    assert mlp.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert mlp.round_bf16(-3.0) == -3.0
    assert mlp.round_bf16(0.0) == 0.0
    x = np.random.default_rng(1).standard_normal(10000) * 10.0 ** np.random.default_rng(2).uniform(-20, 20, 10000)
    r = mlp.round_bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-6))
    assert np.array_equal(mlp.round_bf16(r), r)
    # representable: the low 16 bits of the binary32 encoding are zero
    assert np.all((r.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)


def test_rounded_operands_change_a_product_by_at_most_the_bf16_bound():
    rng = np.random.default_rng(4)
    p = mlp.init_params([6, 5, 3], 7)
    x = rng.standard_normal((4, 6))
    y, _ = mlp.forward(p, x)
    yr, _ = mlp.forward(p, x, mlp.round_bf16)
    # one layer: |dz| <= sum |x||W| * (2^-8 + 2^-8 + 2^-16); the ReLU is 1-Lipschitz
    h = np.abs(x) @ np.abs(p[0])
    bound1 = h * (2 * 2.0 ** -8 + 2.0 ** -16)
    z1 = x @ p[0]
    z1r = mlp.round_bf16(x) @ mlp.round_bf16(p[0])
    assert np.all(np.abs(z1 - z1r) <= bound1 * (1 + 1e-9))
    assert np.max(np.abs(y - yr)) < 0.05 * np.max(np.abs(y))
