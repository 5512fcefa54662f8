"""FP64 oracle of the autotuner's cost model (the MLP of include/bandred_tune.h).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the library.  It shares no
code with the CUDA kernels.

The model is a perceptron with two tanh hidden layers; its parameters sit in one flat
vector in the order W1 (H x D, row-major), b1 (H), W2 (H x H, row-major), b2 (H),
w3 (H), b3 (1).  The loss is the mean squared error.  Gradients are taken by central
finite differences of the loss (no back-propagation here, so the CUDA back-propagation
is checked against an independent route), and Adam follows Kingma & Ba, "Adam: A Method
for Stochastic Optimization" (ICLR 2015), Algorithm 1, with its bias corrections.

Every function works in the dtype of its inputs (float64 normally; complex128 for the
complex-step derivative the tests use as a pin).
"""
from __future__ import annotations

import numpy as np


def param_count(D: int, H: int) -> int:
    return H * D + H + H * H + H + H + 1


def unpack(params: np.ndarray, D: int, H: int):
    """(W1, b1, W2, b2, w3, b3) views of the flat parameter vector."""
    p = np.asarray(params)
    o = 0
    W1 = p[o:o + H * D].reshape(H, D)
    o += H * D
    b1 = p[o:o + H]
    o += H
    W2 = p[o:o + H * H].reshape(H, H)
    o += H * H
    b2 = p[o:o + H]
    o += H
    w3 = p[o:o + H]
    o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(params: np.ndarray, X: np.ndarray, D: int, H: int) -> np.ndarray:
    """y = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3 for every row x of X (rows x D)."""
    W1, b1, W2, b2, w3, b3 = unpack(params, D, H)
    X = np.asarray(X)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3


def loss(params: np.ndarray, X: np.ndarray, t: np.ndarray, D: int, H: int):
    """Mean squared error (1/rows) sum (y - t)^2."""
    e = forward(params, X, D, H) - np.asarray(t)
    return np.mean(e * e)


def fd_grad(params: np.ndarray, X: np.ndarray, t: np.ndarray, D: int, H: int, h: float = 1e-6) -> np.ndarray:
    """Central finite differences (L(p + h e_i) - L(p - h e_i)) / 2h of the loss."""
    p = np.array(params, dtype=np.float64, copy=True)
    g = np.zeros_like(p)
    for i in range(p.size):
        old = p[i]
        p[i] = old + h
        lp = loss(p, X, t, D, H)
        p[i] = old - h
        lm = loss(p, X, t, D, H)
        p[i] = old
        g[i] = (lp - lm) / (2.0 * h)
    return g


def adam_step(params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One step of Adam; returns new (params, m, v)."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return np.asarray(params, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v
