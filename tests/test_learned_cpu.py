"""CPU checks of the learned-guess checkpoints: a saved network (weights, Adam
moments and step count) and a saved step predictor (with its input and output
scalings) load back bit for bit; files of another kind or shape are
rejected.  No GPU calls: the networks live in host memory here."""

import numpy as np
import pytest
import torch

from paper_1008_1700_gb300.learned import GuessNet, StepGuess


def _net(seed=3):
    net = GuessNet(2, 11, hidden=16, layers=2, seed=seed, device="cpu")
    g = torch.Generator().manual_seed(seed)
    net.m.copy_(torch.randn(net.count, generator=g))
    net.v.copy_(torch.rand(net.count, generator=g))
    net.step = 17
    return net


def _same(a, b):
    assert (a.d_in, a.d_out, a.hidden, a.layers, a.count, a.step) == \
        (b.d_in, b.d_out, b.hidden, b.layers, b.count, b.step)
    for k in ("params", "m", "v"):
        assert torch.equal(getattr(a, k), getattr(b, k))


def test_guessnet_checkpoint_round_trip(tmp_path):
    net = _net()
    path = tmp_path / "net.npz"
    net.save(path)
    back = GuessNet.load(path, device="cpu")
    _same(net, back)
    # the loaded network keeps its own buffers
    back.params.add_(1.0)
    assert not torch.equal(back.params, net.params)


def test_step_guess_checkpoint_round_trip(tmp_path):
    g = StepGuess.from_parts(_net(5), b_mean=20.25, b_scale=7.0710678118654755,
                             scale=3.0517578125e-05)
    path = tmp_path / "step.npz"
    g.save(path)
    back = StepGuess.load(path, device="cpu")
    _same(g.net, back.net)
    assert (back.b_mean, back.b_scale, back.scale) == (g.b_mean, g.b_scale, g.scale)


def test_checkpoints_of_another_kind_or_shape_are_rejected(tmp_path):
    net = _net()
    p_net = tmp_path / "net.npz"
    net.save(p_net)
    with pytest.raises(ValueError, match="not a StepGuess checkpoint"):
        StepGuess.load(p_net, device="cpu")
    # a parameter vector of the wrong length
    with np.load(p_net) as z:
        arrays = {k: z[k] for k in z.files}
    arrays["m"] = arrays["m"][:-1]
    p_bad = tmp_path / "bad.npz"
    with open(p_bad, "wb") as f:
        np.savez(f, **arrays)
    with pytest.raises(ValueError, match="array 'm'"):
        GuessNet.load(p_bad, device="cpu")
    # a file without the metadata
    p_none = tmp_path / "none.npz"
    with open(p_none, "wb") as f:
        np.savez(f, params=arrays["params"])
    with pytest.raises(ValueError, match="no checkpoint metadata"):
        GuessNet.load(p_none, device="cpu")
