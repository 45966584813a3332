"""FP64 CPU oracle of the surrogate MLP (test infrastructure).

A plain numpy multilayer perceptron: x -> ReLU(x W0^T + b0) -> ... -> ReLU(. W_{L-1}^T
+ b_{L-1}) -> . W_L^T + b_L, mean squared error over all outputs, analytic
backward pass, and the Adam update.  Only the tests use it, to check the GPU
kernels' forward values, gradients and updates; the GPU path never calls it.

Layers are (W, b) with W of shape (out, in).
"""
from __future__ import annotations

import numpy as np


def init_params(sizes, seed: int):
    """He-normal weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(len(sizes) - 1):
        fan_in = sizes[i]
        W = rng.standard_normal((sizes[i + 1], fan_in)) * np.sqrt(2.0 / fan_in)
        out.append([W, np.zeros(sizes[i + 1])])
    return out


def forward(params, X):
    """Returns (y, activations): activations[i] is the input of layer i."""
    acts = [np.asarray(X, dtype=np.float64)]
    h = acts[0]
    for i, (W, b) in enumerate(params):
        z = h @ W.T + b
        h = np.maximum(z, 0.0) if i < len(params) - 1 else z
        acts.append(h)
    return h, acts


def loss(params, X, Y):
    """Mean squared error over every output of every sample."""
    y, _ = forward(params, X)
    return float(np.mean((y - Y) ** 2))


def gradients(params, X, Y):
    """Analytic gradient of the mean squared error: list of (dW, db)."""
    y, acts = forward(params, X)
    n = y.size
    d = 2.0 * (y - Y) / n
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W, b = params[i]
        h_in = acts[i]
        grads[i] = [d.T @ h_in, d.sum(axis=0)]
        if i > 0:
            d = (d @ W) * (acts[i] > 0.0)
    return grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state = {'t': int, 'm': [...], 'v': [...]}."""
    if not state:
        state["t"] = 0
        state["m"] = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        state["v"] = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
    state["t"] += 1
    t = state["t"]
    for i in range(len(params)):
        for j in range(2):
            g = grads[i][j]
            m = state["m"][i][j] = beta1 * state["m"][i][j] + (1 - beta1) * g
            v = state["v"][i][j] = beta2 * state["v"][i][j] + (1 - beta2) * g * g
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            params[i][j] = params[i][j] - lr * mh / (np.sqrt(vh) + eps)
    return params
