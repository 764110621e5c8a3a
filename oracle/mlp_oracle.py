"""CPU oracle of the warm-start network (test infrastructure only).

Three dense layers with SiLU activations, width W:
    z1 = W1 x + b1, a1 = silu(z1); z2 = W2 a1 + b2, a2 = silu(z2); y = W3 a2 + b3
The weight matrices enter every product rounded to BF16 (round to nearest
even from the FP32 master values); biases, activations and accumulation are
FP64 here (FP32 on the GPU).  Loss: mean over the batch of 1/2 |y - t|^2.
Parameters are one packed vector [W1 | b1 | W2 | b2 | W3 | b3].  This is the
network of the learned fsGW warm start, which the paper does not have.
"""
from __future__ import annotations

import numpy as np


def shapes(d_in, width, d_out):
    return [(width, d_in), (width,), (width, width), (width,), (d_out, width), (d_out,)]


def nparams(d_in, width, d_out):
    return sum(int(np.prod(s)) for s in shapes(d_in, width, d_out))


def unpack(p, d_in, width, d_out):
    out, off = [], 0
    for s in shapes(d_in, width, d_out):
        n = int(np.prod(s))
        out.append(np.asarray(p[off:off + n], dtype=np.float64).reshape(s))
        off += n
    return out


def bf16_round(x):
    """Round FP32 values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, x, d_in, width, d_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, d_in, width, d_out)
    W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    z1 = x @ W1.T + b1
    a1 = silu(z1)
    z2 = a1 @ W2.T + b2
    a2 = silu(z2)
    y = a2 @ W3.T + b3
    return y, (x, z1, a1, z2, a2)


def loss_and_grad(p, x, t, d_in, width, d_out):
    """Loss and its gradient with respect to the packed parameters (the BF16
    rounding of the weights is treated as the identity in the backward pass,
    as in mixed-precision training with FP32 master weights)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, d_in, width, d_out)
    W1r, W2r, W3r = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    y, (x, z1, a1, z2, a2) = forward(p, x, d_in, width, d_out)
    B = x.shape[0]
    dy = (y - t) / B
    loss = 0.5 * np.sum((y - t) ** 2) / B
    gW3 = dy.T @ a2
    gb3 = dy.sum(0)
    da2 = dy @ W3r
    dz2 = da2 * dsilu(z2)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(0)
    da1 = dz2 @ W2r
    dz1 = da1 * dsilu(z1)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g


def init_params(d_in, width, d_out, seed):
    """He-style initialisation (FP32 master values)."""
    g = np.random.default_rng(seed)
    parts = []
    for s in shapes(d_in, width, d_out):
        if len(s) == 2:
            parts.append(g.standard_normal(s) * np.sqrt(1.0 / s[1]))
        else:
            parts.append(np.zeros(s))
    return np.concatenate([a.ravel() for a in parts]).astype(np.float32)


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba) on the FP32 master parameters."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1**step)
    vh = v / (1 - b2**step)
    return (p - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32), m, v
