"""Plain FP64 CPU reference of the proposal MLP (test infrastructure only).

Architecture (the learned-initial-iterate extension of the Newton method of
Section 3.4; the paper itself has no learned component):

    H1 = relu(X W1^T + b1)        X  [B, n_in]
    H2 = relu(H1 W2^T + b2)
    Y  = H2 W3^T + b3              Y  [B, n_out]
    L  = (1/B) sum_b sum_j (Y_bj - T_bj)^2

``forward``/``backward`` follow these formulas with numpy in float64. With
``bf16=True`` the values the GPU stores in bfloat16 (inputs, weights, hidden
activations, the output gradient and the hidden-layer gradients) are rounded
to bfloat16 (round to nearest even) at the same points, so that the CUDA
kernels can be compared with it; every sum is still exact FP64.

Pinned by tests/test_oracle_mlp.py: central finite differences of L in
float64 (bf16=False), and a hand-computed two-unit example.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _r(a, on):
    return bf16_round(a) if on else np.asarray(a, dtype=np.float64)


def forward(X, params, bf16=False):
    W1, b1, W2, b2, W3, b3 = params
    X = _r(X, bf16)
    W1r, W2r, W3r = _r(W1, bf16), _r(W2, bf16), _r(W3, bf16)
    Z1 = X @ W1r.T + b1
    H1 = _r(np.maximum(Z1, 0.0), bf16)
    Z2 = H1 @ W2r.T + b2
    H2 = _r(np.maximum(Z2, 0.0), bf16)
    Y = H2 @ W3r.T + b3
    return Y, (X, W1r, W2r, W3r, H1, H2)


def loss(Y, T):
    return float(np.sum((Y - T) ** 2) / Y.shape[0])


def backward(X, T, params, bf16=False):
    """(L, [dW1, db1, dW2, db2, dW3, db3]) by reverse-mode differentiation."""
    Y, (Xr, W1r, W2r, W3r, H1, H2) = forward(X, params, bf16)
    B = Y.shape[0]
    dY = 2.0 * (Y - T) / B
    db3 = dY.sum(axis=0)
    dYr = _r(dY, bf16)
    dW3 = dYr.T @ H2
    dZ2 = _r((dYr @ W3r) * (H2 > 0), bf16)
    db2 = dZ2.sum(axis=0)
    dW2 = dZ2.T @ H1
    dZ1 = _r((dZ2 @ W2r) * (H1 > 0), bf16)
    db1 = dZ1.sum(axis=0)
    dW1 = dZ1.T @ Xr
    return loss(Y, T), [dW1, db1, dW2, db2, dW3, db3]
