"""Writes ``fullsize_reference.json``: the oracle's solution x = A^-1 f of the
full-size workloads, stored as its 2-norm, its infinity norm and 512 seeded
sampled entries (plus the first and last), for the full-size GPU parity
tests.  Calls only ``oracle/`` (and the input generators in ``workloads``).

* 64^3 slabs and 48^3 sequence steps t = 1, 150: DDPSOracle with a single
  block (p = 1: R = 0, c is empty and Fig. 3 is one exact LU solve, the case
  the oracle pins against LAPACK), SuperLU with the minimum-degree ordering
  of A + A^T (COLAMD's fill on these 3-D grids takes far longer).
* 1M random band: ``jacobi_solution`` (the matrix is strictly diagonally
  dominant by rows: diagonal 1.2 x the off-diagonal absolute row sum) to a
  certified error bound of 1e-15 relative.

Run from the repository root: ``python tests/golden/make_fullsize_reference.py``
(minutes: the 64^3 LU takes the longest)."""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle.ddps_oracle import DDPSOracle, csr, jacobi_solution, relres_inf  # noqa: E402

NSAMPLE = 512
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_reference.json")


def sample_indices(n, seed):
    idx = np.random.default_rng(seed).choice(n, size=NSAMPLE, replace=False)
    return np.unique(np.concatenate([[0, n - 1], idx])).astype(np.int64)


def single_block_lu(P):
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, np.array([0, P.n]), spikes=False,
                   permc_spec="MMD_AT_PLUS_A")
    x, _ = o.precond(P.f)
    return x, o.A


def entry(P, x, A, method, seed, extra=None):
    idx = sample_indices(P.n, seed)
    d = {"n": int(P.n), "method": method, "norm2": float(np.linalg.norm(x)),
         "norm_inf": float(np.max(np.abs(x))), "relres_inf": relres_inf(A, x, P.f),
         "idx": idx.tolist(), "x": [float(v) for v in x[idx]]}
    if extra:
        d.update(extra)
    return d


def main():
    out = {"comment": "oracle x = A^-1 f of the full-size workloads, sampled; written by "
                      "tests/golden/make_fullsize_reference.py"}
    jobs = [("cd3d_48_t1", lambda: W.cfg5(1)), ("cd3d_48_t150", lambda: W.cfg5(150)),
            ("cd3d_64_slabs16", W.cfg2), ("randband_1m", W.cfg4)]
    for k, (name, make) in enumerate(jobs):
        t0 = time.time()
        P = make()
        if name == "randband_1m":
            A = csr(P.n, P.rowptr, P.colind, P.values)
            x, bound = jacobi_solution(A, P.f, tol=1e-15)
            out[name] = entry(P, x, A, "jacobi_solution (certified bound %.2e)" % bound, 100 + k,
                              {"certified_bound_inf": bound})
        else:
            x, A = single_block_lu(P)
            out[name] = entry(P, x, A, "DDPSOracle p=1 (one LU solve, SuperLU MMD_AT_PLUS_A)",
                              100 + k)
        print(name, "%.1f s" % (time.time() - t0), "relres %.2e" % out[name]["relres_inf"],
              flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")


if __name__ == "__main__":
    main()
