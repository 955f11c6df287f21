"""Per-leaf-chunk MLP of the learned right preconditioner (oracle, test
infrastructure).

The network the solver trains on its own residual/error pairs: 128 -> 256 ->
256 -> 128 with ReLU, weights W_l [out][in] and biases b_l.  Storage precision
is BF16 for weights and activations (round to nearest even), arithmetic here
is FP64; with ``bf16=False`` nothing is rounded (used by the finite-difference
pin).  Loss: L = sum over samples and outputs of (y - t)^2 / (2 n).

Parameter vector layout (shared with the library's export): W1, b1, W2, b2,
W3, b3, each row-major.
"""
from __future__ import annotations

import numpy as np

SIZES = (128, 256, 256, 128)


def n_params():
    n = 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        n += a * b + b
    return n


def unpack(theta):
    out, o = [], 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        W = theta[o:o + a * b].reshape(b, a)
        o += a * b
        bb = theta[o:o + b]
        o += b
        out.append((W, bb))
    return out


def bf16(x):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, bf16_store=True):
    """Returns the output and the stored activations [X, H1, H2]."""
    rnd = bf16 if bf16_store else (lambda a: np.asarray(a, np.float64))
    layers = unpack(np.asarray(theta, np.float64))
    acts = [rnd(X)]
    h = acts[0]
    for li, (W, b) in enumerate(layers):
        z = h @ rnd(W).T + b
        if li < len(layers) - 1:
            h = rnd(np.maximum(z, 0.0))
            acts.append(h)
        else:
            h = z
    return h, acts


def loss_grad(theta, X, T, bf16_store=True):
    """MSE loss and its gradient with respect to the parameter vector."""
    rnd = bf16 if bf16_store else (lambda a: np.asarray(a, np.float64))
    layers = unpack(np.asarray(theta, np.float64))
    Y, acts = forward(theta, X, bf16_store)
    n = X.shape[0]
    dY = (Y - T) / n
    loss = 0.5 * np.sum((Y - T) ** 2) / n
    grads = []
    d = dY
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        h = acts[li]
        grads.append((d.T @ h, d.sum(axis=0)))
        if li > 0:
            d = (d @ rnd(W)) * (acts[li] > 0)
    grads = grads[::-1]
    return loss, np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
