"""Helpers shared by the GPU parity tests (CUDA path through the C ABI)."""

import numpy as np
import torch

from paper_1008_1700_gb300 import Solver, native as N

DROP = {None: (N.DDPS_DROP_NONE, 0.0)}


def drop_opts(drop):
    if drop is None:
        return {}
    mode = N.DDPS_DROP_ABS if drop[0] == "abs" else N.DDPS_DROP_COLUMN
    return {"drop_mode": mode, "drop_tol": float(drop[1])}


def make_solver(P, drop=None, **opts):
    o = dict(drop_opts(drop))
    o.update(opts)
    S = Solver(P.rowptr, P.colind, P.block_ptr, values_host=P.values if drop else None, **o)
    S.factor(torch.tensor(P.values, device="cuda"))
    return S


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))
