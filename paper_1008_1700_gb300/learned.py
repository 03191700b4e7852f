"""Learned initial guess for the reduced solve of Fig. 3 (6.3) over a time sequence.

In a time-stepping loop (Fig. 1: time integration around the linear solves)
every step solves a system whose matrix changes smoothly.  DDPS solves the
reduced system G^ z^ = g^ iteratively (6.3), starting from a vector; this
module trains a multilayer perceptron on the reduced solutions that DDPS
produced at earlier steps and uses its prediction as that starting vector.
The inner BiCGStab still runs to its tolerance from the guess, and the solver
drops a guess whose residual is larger than that of zero, so a poor
prediction costs nothing but the prediction itself.

The network's forward pass, backward pass and Adam steps are the library's
kernels (``ddps_mlp_*``); torch only holds the device buffers.

Guess strategies compared by ``run_sequence``:
  ``zero``     z^0 = 0 (the paper's method);
  ``ghat``     z^0 = g^ (drops the coupling term G(c,c));
  ``warm``     z^0 = z^ of the previous step;
  ``mlp``      z^0 = g^ + s * net(beta): the network predicts the coupling
               correction z^ - g^ from the normalised convection coefficient;
  ``mlp_warm`` z^0 = z^_prev + s * net(beta, dbeta): the network predicts the
               change of z^ from one step to the next.
"""

from __future__ import annotations

import json
import math
import time

import numpy as np
import torch

from . import native as N

# Checkpoint format: one ``.npz`` file holding the flat parameter vector, the
# two Adam moment vectors and a JSON string ``meta`` (shape, Adam step count,
# and for ``StepGuess`` its input and output scalings).
_CKPT_FORMAT = "ddps-guessnet-1"


class GuessNet:
    """MLP (``layers`` hidden layers of width ``hidden``, ReLU) on the device."""

    def __init__(self, d_in, d_out, hidden=256, layers=3, seed=0, device="cuda"):
        self.d_in, self.d_out, self.hidden, self.layers = d_in, d_out, hidden, layers
        self.count = N.ddps_mlp_param_count(d_in, hidden, layers, d_out)
        g = torch.Generator(device="cpu").manual_seed(seed)
        dims = [d_in] + [hidden] * layers + [d_out]
        chunks = []
        for l in range(len(dims) - 1):
            bound = math.sqrt(6.0 / dims[l])
            W = (torch.rand(dims[l + 1], dims[l], generator=g) * 2 - 1) * bound
            if l == len(dims) - 2:
                W *= 0.1
            chunks += [W.reshape(-1), torch.zeros(dims[l + 1])]
        self.params = torch.cat(chunks).to(device=device, dtype=torch.float32).contiguous()
        assert self.params.numel() == self.count
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grads = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.step = 0
        self._ws = {}

    def _meta(self):
        return {"format": _CKPT_FORMAT, "d_in": self.d_in, "d_out": self.d_out,
                "hidden": self.hidden, "layers": self.layers, "count": int(self.count),
                "step": int(self.step)}

    def _arrays(self):
        return {k: getattr(self, k).detach().to("cpu", torch.float32).numpy()
                for k in ("params", "m", "v")}

    @classmethod
    def _from_state(cls, meta, arrays, device):
        if meta.get("format") != _CKPT_FORMAT:
            raise ValueError(f"not a GuessNet checkpoint (format {meta.get('format')!r})")
        net = cls(meta["d_in"], meta["d_out"], meta["hidden"], meta["layers"], device=device)
        if net.count != meta["count"]:
            raise ValueError(f"checkpoint holds {meta['count']} parameters, the network "
                             f"has {net.count}")
        for k in ("params", "m", "v"):
            a = np.asarray(arrays[k])
            if a.dtype != np.float32 or a.shape != (net.count,):
                raise ValueError(f"checkpoint array {k!r} has dtype {a.dtype} and shape "
                                 f"{a.shape}, expected float32 ({net.count},)")
            getattr(net, k).copy_(torch.from_numpy(a))
        net.step = int(meta["step"])
        return net

    def save(self, path):
        """Writes the weights, the Adam moments and step count, and the shape
        to ``path`` (one ``.npz`` file), so a later run can predict, or go on
        training, without the training sequence."""
        _write_ckpt(path, self._meta(), self._arrays())

    @classmethod
    def load(cls, path, device="cuda"):
        """The network saved by ``save``, on ``device``."""
        meta, arrays = _read_ckpt(path)
        return cls._from_state(meta, arrays, device)

    def _workspace(self, B):
        if B not in self._ws:
            nb = N.ddps_mlp_workspace_bytes(self.d_in, self.hidden, self.layers, self.d_out, B)
            self._ws[B] = torch.empty(nb, dtype=torch.uint8, device=self.params.device)
        return self._ws[B]

    def forward(self, X):
        X = X.to(torch.float32).contiguous()
        B = X.shape[0]
        Y = torch.empty(B, self.d_out, dtype=torch.float32, device=X.device)
        N.ddps_mlp_forward(self.params, self.d_in, self.hidden, self.layers, self.d_out, X, B, Y,
                           self._workspace(B))
        return Y

    def backward(self, X, T):
        X = X.to(torch.float32).contiguous()
        T = T.to(torch.float32).contiguous()
        B = X.shape[0]
        N.ddps_mlp_backward(self.params, self.d_in, self.hidden, self.layers, self.d_out, X, T, B,
                            self.grads, self.loss, self._workspace(B))
        return self.grads, self.loss

    def fit(self, X, T, iters=2000, lr=1e-3, lr_min=1e-5, beta1=0.9, beta2=0.999, eps=1e-8,
            report=200):
        """Full-batch Adam with a cosine learning-rate decay from ``lr`` to
        ``lr_min``; returns the losses read every ``report`` iterations."""
        losses = []
        for it in range(iters):
            self.backward(X, T)
            self.step += 1
            lr_t = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * it / max(iters - 1, 1)))
            N.ddps_mlp_adam(self.params, self.grads, self.m, self.v, self.count, lr_t, beta1, beta2,
                            eps, self.step)
            if report and (it % report == 0 or it == iters - 1):
                losses.append(float(self.loss.item()))
        return losses


def _write_ckpt(path, meta, arrays):
    with open(path, "wb") as f:
        np.savez(f, meta=np.array(json.dumps(meta, sort_keys=True)), **arrays)


def _read_ckpt(path):
    with np.load(path, allow_pickle=False) as z:
        if "meta" not in z.files:
            raise ValueError(f"{path}: no checkpoint metadata")
        meta = json.loads(str(z["meta"]))
        arrays = {k: z[k] for k in z.files if k != "meta"}
    return meta, arrays


def _beta(b, b_mean, b_scale):
    return (b - b_mean) / b_scale


class StepGuess:
    """The ``mlp_warm`` strategy as a reusable predictor: trained on the
    reduced solutions z^(t) of consecutive steps, it predicts z^(t) from
    z^(t-1) and the normalised coefficients of steps t and t-1."""

    def __init__(self, Z, b, hidden=256, layers=3, seed=1, fit_iters=2000, lr=1e-3):
        b = np.asarray(b, dtype=np.float64)
        self.b_mean = float(b.mean())
        self.b_scale = float(max(b.std(), 1e-12))
        D = Z[1:] - Z[:-1]
        self.scale = float(D.abs().max().item()) or 1.0
        bb = _beta(b, self.b_mean, self.b_scale)
        X = torch.tensor(np.stack([bb[1:], (bb[1:] - bb[:-1]) * 10.0], axis=1),
                         dtype=torch.float32, device=Z.device)
        self.net = GuessNet(2, Z.shape[1], hidden, layers, seed)
        self.losses = self.net.fit(X, (D / self.scale).to(torch.float32), iters=fit_iters, lr=lr)

    @classmethod
    def from_parts(cls, net, b_mean, b_scale, scale):
        """A predictor from a trained network and its scalings (no training)."""
        g = cls.__new__(cls)
        g.net, g.b_mean, g.b_scale, g.scale = net, float(b_mean), float(b_scale), float(scale)
        g.losses = []
        return g

    def save(self, path):
        """Writes the network (as ``GuessNet.save``) and the scalings of its
        input and output to ``path``."""
        meta = self.net._meta()
        meta.update(kind="step_guess", b_mean=self.b_mean, b_scale=self.b_scale,
                    scale=self.scale)
        _write_ckpt(path, meta, self.net._arrays())

    @classmethod
    def load(cls, path, device="cuda"):
        """The predictor saved by ``save``, on ``device``."""
        meta, arrays = _read_ckpt(path)
        if meta.get("kind") != "step_guess":
            raise ValueError(f"{path}: not a StepGuess checkpoint")
        net = GuessNet._from_state(meta, arrays, device)
        return cls.from_parts(net, meta["b_mean"], meta["b_scale"], meta["scale"])

    def predict(self, z_prev, b_t, b_prev):
        bb = _beta(b_t, self.b_mean, self.b_scale)
        bp = _beta(b_prev, self.b_mean, self.b_scale)
        xin = torch.tensor([[bb, (bb - bp) * 10.0]], dtype=torch.float32, device=z_prev.device)
        return (z_prev + self.scale * self.net.forward(xin)[0].to(torch.float64)).contiguous()


def run_sequence(make_problem, coeff, t_train, t_eval, solver_opts, modes=("zero", "mlp"),
                 hidden=256, layers=3, fit_iters=2000, lr=1e-3, seed=0, log=None):
    """Solves the sequence: zero-guess solves on ``t_train`` collect (g^, z^);
    the network is trained; every step of ``t_eval`` is then solved once per
    guess strategy in ``modes``.  Returns a dict of per-mode statistics."""
    from .solver import Solver

    P0 = make_problem(t_train[0])
    S = Solver(P0.rowptr, P0.colind, P0.block_ptr, **solver_opts)
    m = S.m
    dev = "cuda"
    f = torch.tensor(P0.f, device=dev)
    x = torch.empty_like(f)
    zs, gs, bs = [], [], []
    t0 = time.perf_counter()
    for t in t_train:
        P = make_problem(t)
        S.factor(torch.tensor(P.values, device=dev))
        S.set_reduced_guess(None)
        _, info = S.solve(f, x)
        z, g = S.reduced_solution()
        zs.append(z.clone())
        gs.append(g.clone())
        bs.append(coeff(t))
    collect_s = time.perf_counter() - t0

    b_arr = np.array(bs)
    b_mean = float(b_arr.mean())
    b_scale = float(max(b_arr.std(), 1e-12))
    Z = torch.stack(zs)
    G = torch.stack(gs)
    stats = {"m": m, "collect_s": collect_s}
    nets = {}
    t0 = time.perf_counter()
    if "mlp" in modes:
        R = Z - G
        scale = float(R.abs().max().item()) or 1.0
        X = torch.tensor(_beta(b_arr, b_mean, b_scale), dtype=torch.float32, device=dev)[:, None]
        net = GuessNet(1, m, hidden, layers, seed)
        losses = net.fit(X, (R / scale).to(torch.float32), iters=fit_iters, lr=lr)
        nets["mlp"] = (net, scale)
        stats["mlp_losses"] = losses
    if "mlp_warm" in modes:
        D = Z[1:] - Z[:-1]
        scale = float(D.abs().max().item()) or 1.0
        bb = _beta(b_arr, b_mean, b_scale)
        X = torch.tensor(np.stack([bb[1:], (bb[1:] - bb[:-1]) * 10.0], axis=1), dtype=torch.float32,
                         device=dev)
        net = GuessNet(2, m, hidden, layers, seed + 1)
        losses = net.fit(X, (D / scale).to(torch.float32), iters=fit_iters, lr=lr)
        nets["mlp_warm"] = (net, scale)
        stats["mlp_warm_losses"] = losses
    stats["fit_s"] = time.perf_counter() - t0

    res = {mode: {"first_inner": [], "inner": [], "outer": [], "relres": [], "ms": [],
                  "guess_used": []} for mode in modes}
    z_prev = zs[-1]
    b_prev = bs[-1]
    for t in t_eval:
        P = make_problem(t)
        vals = torch.tensor(P.values, device=dev)
        bt = coeff(t)
        z_next = None
        for mode in modes:
            torch.cuda.synchronize()
            tt = time.perf_counter()
            S.factor(vals)
            guess = None
            if mode == "ghat":
                guess = S.reduced_rhs(f)
            elif mode == "warm":
                guess = z_prev
            elif mode == "mlp":
                net, scale = nets["mlp"]
                xin = torch.tensor([[_beta(bt, b_mean, b_scale)]], dtype=torch.float32, device=dev)
                guess = S.reduced_rhs(f) + scale * net.forward(xin)[0].to(torch.float64)
            elif mode == "mlp_warm":
                net, scale = nets["mlp_warm"]
                bb, bp = _beta(bt, b_mean, b_scale), _beta(b_prev, b_mean, b_scale)
                xin = torch.tensor([[bb, (bb - bp) * 10.0]], dtype=torch.float32, device=dev)
                guess = z_prev + scale * net.forward(xin)[0].to(torch.float64)
            S.set_reduced_guess(guess.contiguous() if guess is not None else None)
            _, info = S.solve(f, x)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - tt) * 1e3
            r = res[mode]
            r["first_inner"].append(info["first_inner_iters"])
            r["inner"].append(info["inner_iterations"])
            r["outer"].append(info["outer_iterations"])
            r["relres"].append(info["relres_inf"])
            r["ms"].append(ms)
            r["guess_used"].append(info["guess_used"])
            if mode == modes[0]:
                z_next, _ = S.reduced_solution()
                z_next = z_next.clone()
        z_prev = z_next
        b_prev = bt
        if log:
            log(t, {mode: res[mode]["first_inner"][-1] for mode in modes})
    S.set_reduced_guess(None)
    summary = {}
    for mode in modes:
        r = res[mode]
        summary[mode] = {k: float(np.mean(v)) for k, v in r.items()}
        summary[mode]["relres_max"] = float(np.max(r["relres"]))
    stats["eval"] = summary
    stats["per_step"] = res
    S.close()
    return stats
