"""FP64 reference of the learned cost model (TEST INFRASTRUCTURE ONLY).

The cost model replaces the analytic materialize-versus-recompute estimate of
Eq. 2 (Sec. IV-C) with a small MLP 12 -> 64 -> 64 -> 1 (ReLU).  This file
evaluates the same network in double precision on the same BF16-rounded
values the device kernels use:

  xb = bf(x); a1 = bf(W1) xb + bf(b1); h1 = bf(relu(a1))
  a2 = bf(W2) h1 + bf(b2); h2 = bf(relu(a2)); y = bf(w3) . h2 + bf(b3)
  loss = mean (y - t)^2

bf() rounds to BF16 with round-to-nearest-even.  Gradients are those of the
loss with respect to the FP32 master parameters, treating bf() as the
identity (straight-through), which is what the device backward pass
computes.  Parity with the device is checked in tests; the gradient itself is
pinned by central finite differences of a smooth surrogate in which bf() is
removed (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 12, 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_IN * N_HID
OFF_W2 = OFF_B1 + N_HID
OFF_B2 = OFF_W2 + N_HID * N_HID
OFF_W3 = OFF_B2 + N_HID
OFF_B3 = OFF_W3 + N_HID
N_PARAMS = OFF_B3 + 1


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def unpack(p: np.ndarray):
    p = np.asarray(p)
    W1 = p[OFF_W1:OFF_B1].reshape(N_HID, N_IN)
    b1 = p[OFF_B1:OFF_W2]
    W2 = p[OFF_W2:OFF_B2].reshape(N_HID, N_HID)
    b2 = p[OFF_B2:OFF_W3]
    w3 = p[OFF_W3:OFF_B3]
    b3 = p[OFF_B3]
    return W1, b1, W2, b2, w3, b3


def forward(p: np.ndarray, x: np.ndarray, rounding: bool = True):
    r = bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    pp = np.asarray(p, dtype=np.float32 if rounding else np.float64)
    W1, b1, W2, b2, w3, b3 = (r(v) for v in unpack(pp))
    xb = r(x)
    a1 = xb @ W1.T + b1
    h1 = r(np.maximum(a1, 0.0))
    a2 = h1 @ W2.T + b2
    h2 = r(np.maximum(a2, 0.0))
    y = h2 @ w3 + b3
    return y, (xb, a1, h1, a2, h2, W2, w3)


def loss_grad(p: np.ndarray, x: np.ndarray, t: np.ndarray, rounding: bool = True):
    y, (xb, a1, h1, a2, h2, W2, w3) = forward(p, x, rounding)
    B = len(t)
    d = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(d * d))
    dy = 2.0 * d / B
    g = np.zeros(N_PARAMS)
    g[OFF_W3:OFF_B3] = h2.T @ dy
    g[OFF_B3] = dy.sum()
    da2 = np.outer(dy, w3) * (a2 > 0)
    g[OFF_W2:OFF_B2] = (da2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = da2.sum(0)
    dh1 = da2 @ W2
    da1 = dh1 * (a1 > 0)
    g[OFF_W1:OFF_B1] = (da1.T @ xb).ravel()
    g[OFF_B1:OFF_W2] = da1.sum(0)
    return loss, g
