"""CPU FP64 oracle of the learned-alpha network (TEST INFRASTRUCTURE ONLY).

The network maps spectrum features of g_delta (plus log delta, T and log2 N_t)
to log10(alpha / alpha_rule), alpha_rule the a-priori choice of Section 5
(alpha = delta for PinT-QBVM, tau*delta for PinT-MQBVM):

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = w3 . h2 + b3,
    loss = (1/(2B)) sum_b (y_b - t_b)^2.

Plain numpy, written from the definitions above (chain rule by hand); it
shares nothing with the CUDA kernels.  Pinned by finite differences and by
closed forms in tests/test_mlp_oracle.py.  The paper has no learned component,
so the network's own usefulness is judged by reconstruction error, not parity.
"""
from __future__ import annotations

import numpy as np

__all__ = ["mlp_forward", "mlp_loss_and_grads", "bf16_round", "adam_update"]


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP32 values to bfloat16 (round to nearest even on the top 16 bits),
    returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_forward(params: dict, x: np.ndarray):
    """Returns (y, cache) for a batch x of shape (B, in_dim)."""
    W1, b1, W2, b2, w3, b3 = (np.asarray(params[k], dtype=np.float64) for k in ("W1", "b1", "W2", "b2", "w3", "b3"))
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, (x, z1, h1, z2, h2)


def mlp_loss_and_grads(params: dict, x: np.ndarray, t: np.ndarray):
    """Mean squared error (halved) and its gradient with respect to every parameter."""
    y, (x, z1, h1, z2, h2) = mlp_forward(params, x)
    B = x.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    loss = 0.5 * float(np.mean(r * r))
    dy = r / B                                   # d loss / d y
    w3 = np.asarray(params["w3"], dtype=np.float64)
    W2 = np.asarray(params["W2"], dtype=np.float64)
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array(dy.sum())
    dz2 = np.outer(dy, w3) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adam_update(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) on numpy arrays; returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
