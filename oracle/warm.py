"""Learned warm start: the sketch, the per-row MLP, its loss and gradients (test
infrastructure only).

Not from the paper: the paper initialises players at random (Alg. 2). This is the
warm start of the task: a network maps a random sketch of the first minibatch to an
initial V, and the plain iteration then runs from it.

* Sketch: S = Z^T (Z Omega) / n with Z = [X Y] (n x d, d = d_x + d_y) and a fixed
  Gaussian Omega (d x m); each of the m columns of S is then divided by its root
  mean square over the d rows (feature scaling).
* Network, applied to every row s (m features) of S:
  h1 = relu(W1 s + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3 (o has k entries);
  the d outputs form V0 (d x k). The weights are BF16 values; all arithmetic here is
  FP64.
* Loss of one instance with target V (d x k, the plain solver's solution):
  sum_i (1 - (o_i . v_i)^2 / (|o_i|^2 |v_i|^2)), invariant to the sign and scale of
  every column; a batch of instances averages it.

Pins: tests/test_oracle_warm.py (central finite differences of the loss for every
parameter; sign and scale invariance; zero loss at the target).
"""
from __future__ import annotations

import numpy as np


def sketch(X, Y, omega):
    Z = np.asarray(X, dtype=np.float64) if Y is None else np.hstack([np.asarray(X, np.float64),
                                                                     np.asarray(Y, np.float64)])
    S = Z.T @ (Z @ np.asarray(omega, np.float64)) / Z.shape[0]
    rms = np.sqrt(np.mean(S * S, axis=0))
    return S / rms[None, :]


def forward(params, S):
    W1, b1, W2, b2, W3, b3 = (np.asarray(p, np.float64) for p in params)
    S = np.asarray(S, np.float64)
    z1 = S @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    o = h2 @ W3.T + b3
    return o, (S, z1, h1, z2, h2)


def loss_instance(O, V):
    O = np.asarray(O, np.float64)
    V = np.asarray(V, np.float64)
    c = np.sum(O * V, axis=0)
    a = np.sum(O * O, axis=0)
    t = np.sum(V * V, axis=0)
    return float(np.sum(1.0 - c * c / (a * t)))


def loss_and_grads(params, S_list, V_list):
    """Mean loss over instances and its gradients with respect to every parameter."""
    W1, b1, W2, b2, W3, b3 = (np.asarray(p, np.float64) for p in params)
    grads = [np.zeros_like(W1), np.zeros_like(b1), np.zeros_like(W2), np.zeros_like(b2), np.zeros_like(W3),
             np.zeros_like(b3)]
    total = 0.0
    n = len(S_list)
    for S, V in zip(S_list, V_list):
        O, (Sx, z1, h1, z2, h2) = forward(params, S)
        V = np.asarray(V, np.float64)
        c = np.sum(O * V, axis=0)
        a = np.sum(O * O, axis=0)
        t = np.sum(V * V, axis=0)
        total += float(np.sum(1.0 - c * c / (a * t)))
        # d loss / d o_ri = (2 c_i / (a_i t_i)) (c_i o_ri / a_i - v_ri)
        dO = (2.0 * c / (a * t))[None, :] * (c[None, :] * O / a[None, :] - V) / n
        grads[4] += dO.T @ h2
        grads[5] += dO.sum(axis=0)
        dh2 = (dO @ W3) * (z2 > 0)
        grads[2] += dh2.T @ h1
        grads[3] += dh2.sum(axis=0)
        dh1 = (dh2 @ W2) * (z1 > 0)
        grads[0] += dh1.T @ Sx
        grads[1] += dh1.sum(axis=0)
    return total / n, grads
