"""The learned-guess network's CUDA kernels (forward, backward, Adam) against
the FP64 oracle network on the same parameters and data."""

import numpy as np
import pytest
import torch

from oracle import mlp_oracle as M
from paper_1008_1700_gb300 import native as N

pytestmark = pytest.mark.gpu


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def _setup(seed, d_in=3, hidden=16, layers=3, d_out=20, B=6):
    rng = np.random.default_rng(seed)
    params = M.init_params(d_in, d_out, hidden=hidden, layers=layers, seed=seed)
    params = [(W + 0.05 * rng.standard_normal(W.shape), b + 0.1 * rng.standard_normal(b.shape))
              for W, b in params]
    X = rng.standard_normal((B, d_in))
    T = rng.standard_normal((B, d_out))
    return params, X, T, (d_in, hidden, layers, d_out, B)


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_forward_and_gradients_match_oracle(seed):
    params, X, T, (d_in, hidden, layers, d_out, B) = _setup(seed)
    p = _dev(_flat(params))
    assert p.numel() == N.ddps_mlp_param_count(d_in, hidden, layers, d_out)
    ws = torch.empty(N.ddps_mlp_workspace_bytes(d_in, hidden, layers, d_out, B), dtype=torch.uint8,
                     device="cuda")
    Y = torch.empty(B, d_out, dtype=torch.float32, device="cuda")
    N.ddps_mlp_forward(p, d_in, hidden, layers, d_out, _dev(X), B, Y, ws)
    Yo, _ = M.forward(params, X)
    assert np.max(np.abs(Y.cpu().numpy() - Yo)) <= 1e-5 * max(1.0, np.max(np.abs(Yo)))
    g = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    N.ddps_mlp_backward(p, d_in, hidden, layers, d_out, _dev(X), _dev(T), B, g, loss, ws)
    go = _flat(M.backward(params, X, T))
    gg = g.cpu().numpy()
    assert np.linalg.norm(gg - go) <= 1e-5 * np.linalg.norm(go)
    assert abs(loss.item() - M.loss(params, X, T)) <= 1e-5 * M.loss(params, X, T)


def test_adam_matches_oracle():
    params, X, T, (d_in, hidden, layers, d_out, B) = _setup(5)
    p = _dev(_flat(params))
    state = {}
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    for step in (1, 2, 3):
        grads = M.backward(params, X, T)
        g = _dev(_flat(grads))
        N.ddps_mlp_adam(p, g, m, v, p.numel(), 1e-2, 0.9, 0.999, 1e-8, step)
        M.adam_step(params, grads, state, lr=1e-2)
    assert np.max(np.abs(p.cpu().numpy() - _flat(params))) <= 1e-5
