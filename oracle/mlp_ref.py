"""CPU reference of the ordering network (not in the paper): forward pass,
masked binary cross-entropy loss and gradients, in plain numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  It follows the network's
definition step by step: two hidden layers of H units with ReLU and a linear
output layer,

    H1 = relu(X W1 + b1),  H2 = relu(H1 W2 + b2),  Y = H2 W3 + b3,
    loss = sum over rows r, outputs o of M[r,o] * bce(Y[r,o], T[r,o]) / rows,
    bce(y, t) = max(y, 0) - y t + log(1 + exp(-|y|)),

and its gradients by the chain rule (dY = M (sigmoid(Y) - T) / rows, then
back through the layers).  The device computes with bf16 operands and fp32
accumulation; `quantised=True` rounds, at exactly the same places, the inputs,
weights, hidden activations and back-propagated errors to bf16 (round to
nearest even) so that the two agree up to the order of fp32 summation.
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


def _q(quantised):
    # bf16 rounding for the device-matching path; float64 for the exact one
    return bf16 if quantised else (lambda x: np.asarray(x, dtype=np.float64))


def forward(params, X, quantised=True):
    W1, b1, W2, b2, W3, b3 = params
    q = _q(quantised)
    Xq = q(X)
    Z1 = Xq @ q(W1) + b1
    H1 = q(np.maximum(Z1, 0.0))
    Z2 = H1 @ q(W2) + b2
    H2 = q(np.maximum(Z2, 0.0))
    Y = H2 @ q(W3) + b3
    return (Y.astype(np.float32) if quantised else Y), (Xq, H1, H2)


def loss_and_grads(params, X, T, M, quantised=True):
    """Masked mean BCE over rows and its gradients [dW1, db1, dW2, db2, dW3, db3]."""
    W1, b1, W2, b2, W3, b3 = params
    q = _q(quantised)
    rows = X.shape[0]
    Y, (Xq, H1, H2) = forward(params, X, quantised)
    bce = np.maximum(Y, 0) - Y * T + np.log1p(np.exp(-np.abs(Y)))
    loss = float((M * bce).sum() / rows)
    sig = 1.0 / (1.0 + np.exp(-Y))
    dY = M * (sig - T) / rows
    if quantised:
        dY = dY.astype(np.float32)
    dYq = q(dY)
    dW3 = H2.T @ dYq
    db3 = dY.sum(axis=0)
    dH2 = (dYq @ q(W3).T) * (H2 > 0)
    dH2q = q(dH2)
    dW2 = H1.T @ dH2q
    db2 = dH2.sum(axis=0)
    dH1 = (dH2q @ q(W2).T) * (H1 > 0)
    dH1q = q(dH1)
    dW1 = Xq.T @ dH1q
    db1 = dH1.sum(axis=0)
    grads = (dW1, db1, dW2, db2, dW3, db3)
    return loss, [g.astype(np.float32) if quantised else g for g in grads]
