"""FP64 CPU oracle of the learned initial-guess network (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module; it shares no code with the CUDA kernels it checks.

The network maps a feature vector to a prediction for the reduced unknowns
z^ of Fig. 3 step 6.3 (the paper solves that system iteratively; its initial
guess is the hook the network fills).  Architecture, loss and optimiser are
textbook definitions written out plainly:

* multilayer perceptron, three hidden layers of width H with ReLU, linear
  output:  a_0 = x,  z_l = W_l a_{l-1} + b_l,  a_l = max(z_l, 0) (l = 1..3),
  y = W_4 a_3 + b_4; W_l is stored row-major [out x in];
* loss  L = (1 / (2B)) * sum_b ||y_b - t_b||_2^2  over a batch of B rows;
* gradients by the chain rule (backpropagation);
* Adam (Kingma & Ba, 2015) with bias correction:
  m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
  theta <- theta - lr * (m / (1-b1^k)) / (sqrt(v / (1-b2^k)) + eps).

Pins: central finite differences of ``loss`` against ``backward`` on a small
net; Adam's first step against its closed form -lr g / (|g| + eps); a net whose
hidden layers are forced into their linear region reproduces a plain affine
map.
"""

from __future__ import annotations

import numpy as np


def init_params(d_in: int, d_out: int, hidden: int = 256, layers: int = 3, seed: int = 0):
    """He-uniform weights, zero biases; returns a list [(W1, b1), ..., (W4, b4)]."""
    rng = np.random.default_rng(seed)
    dims = [d_in] + [hidden] * layers + [d_out]
    params = []
    for l in range(len(dims) - 1):
        fan_in = dims[l]
        bound = np.sqrt(6.0 / fan_in)
        W = rng.uniform(-bound, bound, (dims[l + 1], dims[l]))
        if l == len(dims) - 2:
            W *= 0.1
        params.append((W, np.zeros(dims[l + 1])))
    return params


def forward(params, X):
    """Returns the output Y [B x d_out] and the cache of activations."""
    a = np.asarray(X, dtype=np.float64)
    acts = [a]
    pre = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = a @ W.T + b
        pre.append(z)
        a = np.maximum(z, 0.0) if l < L - 1 else z
        acts.append(a)
    return a, (acts, pre)


def loss(params, X, T):
    Y, _ = forward(params, X)
    B = X.shape[0]
    return 0.5 * float(np.sum((Y - T) ** 2)) / B


def backward(params, X, T):
    """Gradients [(dW1, db1), ...] of ``loss`` by backpropagation."""
    Y, (acts, pre) = forward(params, X)
    B = X.shape[0]
    d = (Y - T) / B
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        grads[l] = (d.T @ acts[l], d.sum(axis=0))
        if l > 0:
            d = (d @ W) * (pre[l - 1] > 0.0)
    return grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; ``state`` is {"k": int, "m": [...], "v": [...]}."""
    if not state:
        state["k"] = 0
        state["m"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        state["v"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    state["k"] += 1
    k = state["k"]
    new = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out = []
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            m = state["m"][l][j]
            v = state["v"][l][j]
            m[...] = b1 * m + (1 - b1) * g
            v[...] = b2 * v + (1 - b2) * g * g
            mhat = m / (1 - b1 ** k)
            vhat = v / (1 - b2 ** k)
            out.append(p - lr * mhat / (np.sqrt(vhat) + eps))
        new.append(tuple(out))
    for l in range(len(params)):
        params[l] = new[l]
    return params
