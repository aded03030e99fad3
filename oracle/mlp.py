"""FP64 reference of the warm-start network (TEST INFRASTRUCTURE ONLY).

6 -> 64 -> 64 -> 1 multilayer perceptron with SiLU activations, flat parameter vector
[W1 (64x6), b1 (64), W2 (64x64), b2 (64), W3 (64), b3 (1)] and normalisation
[feature means (6), feature std (6), target mean, target std]. Loss: mean over the batch
of (y - t)^2 / 2 on the normalised target t = (log10 T_d - mean) / std.

With bf16=True the weights and each layer's input are rounded to BF16 (round to
nearest even, written out below from the format's definition: 1 sign, 8 exponent and 7
fraction bits), as the GPU kernels multiply them; gradients then treat the rounding as
the identity (straight through). With bf16=False everything stays FP64, which is the
smooth function the finite-difference pins check.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 6, 64
O_W1, O_B1 = 0, 384
O_W2, O_B2 = 448, 4544
O_W3, O_B3 = 4608, 4672
N_PARAMS = 4673


def bf16_round(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[O_W1:O_B1].reshape(N_HID, N_IN), p[O_B1:O_W2], p[O_W2:O_B2].reshape(N_HID, N_HID),
            p[O_B2:O_W3], p[O_W3:O_B3], p[O_B3])


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, norm, X, bf16=True):
    """Normalised prediction y and the intermediates (a0, z1, a1, z2, a2)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    norm = np.asarray(norm, dtype=np.float64)
    r = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    if bf16:
        W1, W2, W3 = r(W1), r(W2), r(W3)
    xn = (np.asarray(X, dtype=np.float64) - norm[0:6]) / norm[6:12]
    a0 = r(xn.astype(np.float32)) if bf16 else xn
    z1 = a0 @ W1.T + b1
    a1 = r(silu(z1).astype(np.float32)) if bf16 else silu(z1)
    z2 = a1 @ W2.T + b2
    a2 = r(silu(z2).astype(np.float32)) if bf16 else silu(z2)
    y = a2 @ W3 + b3
    return y, (a0, z1, a1, z2, a2)


def predict_log10(p, norm, X, bf16=True):
    y, _ = forward(p, norm, X, bf16)
    return y * norm[13] + norm[12]


def loss_and_grad(p, norm, X, logT, bf16=True):
    """Mean loss and its gradient with respect to the flat parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    if bf16:
        W2, W3 = bf16_round(W2), bf16_round(W3)
    norm = np.asarray(norm, dtype=np.float64)
    y, (a0, z1, a1, z2, a2) = forward(p, norm, X, bf16)
    t = (np.asarray(logT, dtype=np.float64) - norm[12]) / norm[13]
    B = len(t)
    loss = 0.5 * np.mean((y - t) ** 2)
    dy = (y - t) / B
    g = np.zeros(N_PARAMS)
    g[O_W3:O_B3] = dy @ a2
    g[O_B3] = dy.sum()
    dz2 = np.outer(dy, W3) * dsilu(z2)
    g[O_W2:O_B2] = (dz2.T @ a1).reshape(-1)
    g[O_B2:O_W3] = dz2.sum(0)
    dz1 = (dz2 @ W2) * dsilu(z1)
    g[O_W1:O_B1] = (dz1.T @ a0).reshape(-1)
    g[O_B1:O_W2] = dz1.sum(0)
    return loss, g
