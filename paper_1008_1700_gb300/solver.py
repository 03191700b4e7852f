"""Convenience wrapper over the C ABI for PyTorch callers.

``Solver`` owns one ``ddps_handle``: the symbolic analysis of one system, or
of a batch of independent systems stacked block-diagonally.  Values,
right-hand sides and solutions are CUDA float64 tensors; all arithmetic runs
in the library's kernels.
"""

from __future__ import annotations

import numpy as np

from . import native as N


def stack_systems(systems):
    """Stack independent CSR systems into one block-diagonal pattern.

    ``systems`` yields (rowptr, colind, values, block_ptr) tuples.  Returns
    (rowptr, colind, values, block_ptr, sys_block_ptr, sys_row_ptr)."""
    rps, cis, vals, bps = [], [], [], []
    sbp, srp = [0], [0]
    row_off = nnz_off = 0
    for rowptr, colind, values, block_ptr in systems:
        rowptr = np.asarray(rowptr, dtype=np.int64)
        n = len(rowptr) - 1
        rps.append(rowptr[:-1] + nnz_off)
        cis.append(np.asarray(colind, dtype=np.int64) + row_off)
        vals.append(np.asarray(values, dtype=np.float64))
        bps.append(np.asarray(block_ptr, dtype=np.int64)[:-1] + row_off)
        row_off += n
        nnz_off += int(rowptr[-1])
        sbp.append(sbp[-1] + len(block_ptr) - 1)
        srp.append(row_off)
    rowptr = np.concatenate(rps + [np.array([nnz_off])]).astype(np.int32)
    colind = np.concatenate(cis).astype(np.int32)
    block_ptr = np.concatenate(bps + [np.array([row_off])]).astype(np.int64)
    return (rowptr, colind, np.concatenate(vals), block_ptr,
            np.asarray(sbp, dtype=np.int32), np.asarray(srp, dtype=np.int64))


class Solver:
    """One analysed (batch of) system(s)."""

    def __init__(self, rowptr, colind, block_ptr, sys_block_ptr=None, values_host=None,
                 **options):
        self.options = N.default_options(**options)
        self.h = N.ddps_analyze(rowptr, colind, block_ptr, sys_block_ptr, values_host, self.options)
        self.sizes = N.ddps_get_sizes(self.h)
        self.n = self.sizes["n"]
        self.m = self.sizes["m"]

    @classmethod
    def from_systems(cls, systems, **options):
        rowptr, colind, values, block_ptr, sbp, srp = stack_systems(systems)
        needs_values = options.get("drop_mode", 0) != N.DDPS_DROP_NONE
        s = cls(rowptr, colind, block_ptr, sbp, values if needs_values else None, **options)
        s.sys_row_ptr = srp
        s.values_host = values
        return s

    def factor(self, values):
        """Fig. 2 steps 1-5 with new values: a CUDA tensor, or host memory (a
        NumPy array or a CPU tensor), which is copied through the C ABI."""
        if isinstance(values, np.ndarray) or not getattr(values, "is_cuda", False):
            N.ddps_factor_host(self.h, np.ascontiguousarray(values, dtype=np.float64)
                               if isinstance(values, np.ndarray) else values)
        else:
            N.ddps_factor(self.h, values)

    def solve(self, f, x=None, x0=None):
        """f: CUDA tensor (n,) or (nrhs, n); x0: initial guesses of the same
        shape or None (x0 = 0)."""
        import torch
        if x is None:
            x = torch.empty_like(f)
        st, info = N.ddps_solve(self.h, f, x, x0)
        info["status"] = N.STATUS[st]
        return x, info

    def solve_host(self, f, x0=None, x=None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if x is None:
            x = np.empty_like(f)
        if x0 is not None:
            x0 = np.ascontiguousarray(x0, dtype=np.float64)
        st, info = N.ddps_solve_host(self.h, f, x, x0)
        info["status"] = N.STATUS[st]
        return x, info

    def block_solve(self, y):
        import torch
        g = torch.empty_like(y)
        N.ddps_block_solve(self.h, y, g)
        return g

    def reduced_rhs(self, y):
        import torch
        g = torch.empty(self.m, dtype=torch.float64, device=y.device)
        N.ddps_reduced_rhs(self.h, y, g)
        return g

    def reduced_matvec(self, v):
        import torch
        w = torch.empty_like(v)
        N.ddps_reduced_matvec(self.h, v, w)
        return w

    def reduced_solve(self, ghat):
        import torch
        z = torch.empty_like(ghat)
        N.ddps_reduced_solve(self.h, ghat, z)
        return z

    def precond_apply(self, y):
        import torch
        z = torch.empty_like(y)
        N.ddps_precond_apply(self.h, y, z)
        return z

    def spmv(self, x):
        import torch
        y = torch.empty_like(x)
        N.ddps_spmv(self.h, x, y)
        return y

    def set_reduced_guess(self, zhat0):
        N.ddps_set_reduced_guess(self.h, zhat0)

    def reduced_solution(self):
        import torch
        z = torch.empty(self.m, dtype=torch.float64, device="cuda")
        g = torch.empty(self.m, dtype=torch.float64, device="cuda")
        N.ddps_get_reduced_solution(self.h, z, g)
        return z, g

    def tuning(self):
        return N.ddps_get_tuning(self.h)

    def interface(self):
        return N.ddps_get_interface(self.h)

    def ghat_layout(self, b):
        return N.ddps_get_ghat_layout(self.h, b)

    def ghat_block(self, b):
        return N.ddps_get_ghat_block(self.h, b)

    def set_profiling(self, mask):
        N.ddps_set_profiling(self.h, mask)

    def profile(self, reset=True):
        return N.ddps_get_profile(self.h, reset)

    def launch_count(self):
        return N.ddps_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            N.ddps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
