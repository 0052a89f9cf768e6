"""FP64 reference of the mass-preconditioner network (test infrastructure).

A plain multilayer perceptron, written from the textbook definitions, that the
CUDA library's BF16 kernels are checked against:

    h1 = relu(x W1 + b1),  h2 = relu(h1 W2 + b2),  y = h2 W3 + b3
    loss = (1/(B * n_out)) sum (y - t)^2                  (mean squared error)

Backpropagation by the chain rule; Adam (Kingma & Ba 2015) with bias
correction.  Weights W_l are [n_in, n_out] row-major, biases [n_out].

`rnd`, if given, is applied to both operands of every matrix product (with
round_bf16 it states the operand precision of a BF16 tensor-core product while
the sums stay FP64).

The paper has no network: its HMC uses the diagonal Fourier mass of Eq.
Mass_matrix and notes that the mass affects only efficiency, not validity
(Sec. 4.1.2).  The network predicts per-bin log multipliers of that mass.
"""
import numpy as np


def relu(x):
    return np.maximum(x, 0.0)


def init_params(sizes, seed):
    """He-style uniform init: W ~ U(-sqrt(6/n_in), sqrt(6/n_in)), b = 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / n_in)
        params.append(rng.uniform(-lim, lim, size=(n_in, n_out)))
        params.append(np.zeros(n_out))
    return params


def round_bf16(x):
    """Round to the nearest bfloat16 value, ties to even (bfloat16 keeps the sign,
    the 8 exponent bits and the 7 leading fraction bits of a binary32 number).
    Finite inputs only; the result is returned as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(a):
    return a


def forward(params, x, rnd=None):
    """Returns (y, cache)."""
    rnd = rnd or _ident
    acts = [np.asarray(x, dtype=np.float64)]
    zs = []
    n_layers = len(params) // 2
    h = acts[0]
    for l in range(n_layers):
        W, b = params[2 * l], params[2 * l + 1]
        z = rnd(h) @ rnd(W) + b
        zs.append(z)
        h = relu(z) if l < n_layers - 1 else z
        acts.append(h)
    return h, (acts, zs)


def loss_and_grad(params, x, t, rnd=None):
    """MSE loss and its gradient with respect to every parameter."""
    rnd = rnd or _ident
    y, (acts, zs) = forward(params, x, rnd)
    B, n_out = y.shape
    loss = np.sum((y - t) ** 2) / (B * n_out)
    g = 2.0 * (y - t) / (B * n_out)
    n_layers = len(params) // 2
    grads = [None] * len(params)
    for l in reversed(range(n_layers)):
        W = params[2 * l]
        grads[2 * l] = rnd(acts[l]).T @ rnd(g)
        grads[2 * l + 1] = g.sum(axis=0)
        if l > 0:
            g = (rnd(g) @ rnd(W).T) * (zs[l - 1] > 0)
    return loss, grads


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (in place on params, m, v); `step` counts from 1."""
    for i in range(len(params)):
        m[i] = beta1 * m[i] + (1.0 - beta1) * grads[i]
        v[i] = beta2 * v[i] + (1.0 - beta2) * grads[i] ** 2
        mh = m[i] / (1.0 - beta1 ** step)
        vh = v[i] / (1.0 - beta2 ** step)
        params[i] = params[i] - lr * mh / (np.sqrt(vh) + eps)
    return params, m, v
