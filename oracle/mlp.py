"""FP64 reference of the step-controller network (oracle; test infrastructure only).

A three-layer perceptron y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3 with hidden width
128, trained with a weighted mean-squared error and Adam.  This is the plain
textbook definition (backpropagation by the chain rule; Adam as published by
Kingma and Ba, 2015) used to check the GPU training and inference kernels.
The paper itself has no network: the controller is an addition of this
implementation (the paper names adaptive stepping as future work, Sec. 6).

Parameter layout (shared with the GPU kernels' contract): W_l is (out x in),
row-major; biases are vectors.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 128


def init_params(n_in: int, n_out: int, rng: np.random.Generator, hidden: int = HIDDEN):
    """Glorot-uniform weights, zero biases."""
    def glorot(o, i):
        lim = np.sqrt(6.0 / (i + o))
        return rng.uniform(-lim, lim, size=(o, i))
    return {"W1": glorot(hidden, n_in), "b1": np.zeros(hidden),
            "W2": glorot(hidden, hidden), "b2": np.zeros(hidden),
            "W3": glorot(n_out, hidden), "b3": np.zeros(n_out)}


def forward(p, X):
    """X: (B, n_in) -> (Y, cache)."""
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = np.tanh(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.tanh(Z2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (X, H1, H2)


def loss(p, X, T, w=None):
    """(1 / 2B) sum_b sum_o w_o (y_bo - t_bo)^2."""
    Y, _ = forward(p, X)
    w = np.ones(Y.shape[1]) if w is None else np.asarray(w, dtype=np.float64)
    return 0.5 * float(np.sum(w[None, :] * (Y - T) ** 2)) / X.shape[0]


def grads(p, X, T, w=None):
    """Gradients of `loss` by the chain rule."""
    Y, (X, H1, H2) = forward(p, X)
    B = X.shape[0]
    w = np.ones(Y.shape[1]) if w is None else np.asarray(w, dtype=np.float64)
    dY = (Y - T) * w[None, :] / B
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dZ2 = (dY @ p["W3"]) * (1.0 - H2 ** 2)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(0)
    dZ1 = (dZ2 @ p["W2"]) * (1.0 - H1 ** 2)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(0)
    return g


def adam_step(p, g, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v (dicts) and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m", {}).setdefault(k, np.zeros_like(p[k]))
        v = state.setdefault("v", {}).setdefault(k, np.zeros_like(p[k]))
        m *= beta1
        m += (1 - beta1) * g[k]
        v *= beta2
        v += (1 - beta2) * g[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)
    return p
