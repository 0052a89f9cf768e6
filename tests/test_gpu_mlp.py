"""The network kernels (BF16 operands, FP32 accumulation) against the oracle
network: forward, loss, every parameter gradient, and the Adam update.

Two references.  (1) The oracle with every matrix-product operand rounded to
BF16 (round_bf16) and FP64 sums: the kernels take the same operand precision
decisions and differ only by FP32 accumulation order and rare rounding flips
of FP32 intermediates, relative L2 <= 2e-3.  (2) The plain FP64 oracle: BF16
keeps 8 significant bits (operand error <= 2^-9 relative), and backpropagation
through three layers compounds it with cancellation in the sums; the measured
error is about 2e-2 for the first-layer weight gradient, checked at 6e-2."""
import numpy as np
import pytest

from oracle import mlp
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

SIZES = [32, 128, 128, 64]


def problem(seed=0, B=300):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(SIZES, seed + 1)
    for i in range(1, len(params), 2):
        params[i] = rng.standard_normal(params[i].shape) * 0.05
    x = rng.standard_normal((B, SIZES[0]))
    t = rng.standard_normal((B, SIZES[-1])) * 0.5
    return params, x, t


def test_forward_loss_and_gradients_match_oracle():
    import torch

    from paper_1306_1821_gb300 import bps
    params, x, t = problem()
    net = bps.MLP(SIZES)
    try:
        net.set_params(bps.flatten_params(params))
        p32 = bps.unflatten_params(net.get_params(), SIZES)     # the FP32 values the GPU holds
        xs = torch.from_numpy(x.astype(np.float32)).cuda()
        ts = torch.from_numpy(t.astype(np.float32)).cuda()
        y = torch.zeros((x.shape[0], SIZES[-1]), dtype=torch.float32, device="cuda")
        net.forward(xs, y)
        x64 = x.astype(np.float32).astype(np.float64)
        t64 = t.astype(np.float32).astype(np.float64)
        yb, _ = mlp.forward(p32, x64, mlp.round_bf16)
        yr, _ = mlp.forward(p32, x64)
        assert rel_l2(y.cpu().numpy(), yb) < 2e-3
        assert rel_l2(y.cpu().numpy(), yr) < 6e-2
        loss, g = net.loss_grad(xs, ts)
        lb, gb = mlp.loss_and_grad(p32, x64, t64, mlp.round_bf16)
        lr, gr = mlp.loss_and_grad(p32, x64, t64)
        assert loss == pytest.approx(lb, rel=2e-3)
        assert loss == pytest.approx(lr, rel=6e-2)
        gs = bps.unflatten_params(g, SIZES)
        for a, b, c in zip(gs, gb, gr):
            assert rel_l2(a, b) < 2e-3
            assert rel_l2(a, c) < 6e-2
    finally:
        net.close()


def test_adam_step_matches_oracle_update():
    import torch

    from paper_1306_1821_gb300 import bps
    params, x, t = problem(3, 64)
    net = bps.MLP(SIZES)
    try:
        net.set_params(bps.flatten_params(params))
        p0 = bps.unflatten_params(net.get_params(), SIZES)
        xs = torch.from_numpy(x.astype(np.float32)).cuda()
        ts = torch.from_numpy(t.astype(np.float32)).cuda()
        _, g = net.loss_grad(xs, ts)
        net.adam_step(1e-3)
        p1 = bps.unflatten_params(net.get_params(), SIZES)
        gs = bps.unflatten_params(g, SIZES)
        m = [np.zeros_like(q) for q in p0]
        v = [np.zeros_like(q) for q in p0]
        ref = [q.copy() for q in p0]
        mlp.adam_step(ref, gs, m, v, 1, 1e-3)
        for a, b in zip(p1, ref):
            assert np.max(np.abs(a - b)) < 1e-6
    finally:
        net.close()


def test_training_reduces_the_loss():
    import torch

    from paper_1306_1821_gb300 import bps
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, size=(2048, SIZES[0]))
    w = rng.standard_normal((SIZES[0], SIZES[-1])) / np.sqrt(SIZES[0])
    t = np.tanh(x @ w) + 0.5 * np.sin(2 * x[:, :1])
    net = bps.MLP(SIZES)
    try:
        net.set_params(bps.flatten_params(mlp.init_params(SIZES, 11)))
        xs = torch.from_numpy(x.astype(np.float32)).cuda()
        ts = torch.from_numpy(t.astype(np.float32)).cuda()
        l0, _ = net.loss_grad(xs, ts)
        net.train(xs, ts, batch=128, steps=1500, lr=2e-3, seed=5)
        l1, _ = net.loss_grad(xs, ts)
        assert l1 < 0.1 * l0, (l0, l1)
    finally:
        net.close()
