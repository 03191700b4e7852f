"""Edge cases of the method through the C ABI, against the oracle or LAPACK:
one block (c is empty and Fig. 3 is one LU solve), everything dropped (c is
empty, DDPS is block Jacobi inside the Krylov loop), ragged partitions with
one-row blocks, a tiny system, the identity, and batches that mix these."""

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from gpu_helpers import dev, host, make_solver, relerr
from oracle.ddps_oracle import DDPSOracle
from paper_1008_1700_gb300 import Solver, native as N

pytestmark = pytest.mark.gpu

FP64 = dict(factor_prec=N.DDPS_FP64, spike_prec=N.DDPS_FP64, ghat_prec=N.DDPS_FP64,
            inner_prec=N.DDPS_FP64)
MIXED_TC = dict(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_BF16X3, ghat_prec=N.DDPS_FP16,
                inner_prec=N.DDPS_FP32, update_prec=N.DDPS_BF16X3)


def _problem(A, block_ptr, seed=0):
    A = sp.csr_matrix(A)
    A.sort_indices()
    x = np.random.default_rng(seed).uniform(-1, 1, A.shape[0])
    return W.Problem(n=A.shape[0], rowptr=A.indptr.astype(np.int32),
                     colind=A.indices.astype(np.int32), values=A.data.astype(np.float64),
                     block_ptr=np.asarray(block_ptr, dtype=np.int64), f=A @ x, x_true=x)


def _check_solve(P, opts, drop=None, tol=1e-12, max_outer=None):
    S = make_solver(P, drop, tol_out=tol, tol_in=1e-8, maxit_in=300, **opts)
    x, info = S.solve(dev(P.f))
    assert info["status"] == "DDPS_OK", info
    x = host(x)
    A = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, spikes=False).A
    assert np.max(np.abs(P.f - A @ x)) / np.max(np.abs(P.f)) <= tol
    assert relerr(x, np.linalg.solve(A.toarray(), P.f)) <= 1e-8
    if max_outer is not None:
        assert info["outer_iterations"] <= max_outer
    return S, info


@pytest.mark.parametrize("opts", [FP64, MIXED_TC], ids=["fp64", "mixed"])
def test_single_block_is_one_lu_solve(opts):
    """p = 1: R = 0, c is empty; the preconditioner is the (FP64) LU solve, so
    FP64 converges at the first half step; reduced calls accept m = 0."""
    P = W.small_random_band(800, 1, 60, seed=5)
    S, info = _check_solve(P, opts, max_outer=0.5 if opts is FP64 else 3.0)
    assert S.m == 0 and info["inner_iterations"] == 0
    assert S.sizes["ghat_entries"] == 0
    S.close()


def test_everything_dropped_is_block_jacobi():
    """A drop threshold above every entry of R: c is empty, P = D~, and the
    outer Krylov iteration alone couples the blocks."""
    P = W.small_random_band(1500, 6, 100, seed=6)
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, drop=("abs", 1e9))
    assert o.m == 0
    S, info = _check_solve(P, FP64, drop=("abs", 1e9))
    assert S.m == 0 and info["outer_iterations"] > 1.0
    xo, oinfo = o.solve(P.f, tol=1e-12)
    assert abs(info["outer_iterations"] - oinfo["iterations"]) <= 1.0
    S.close()


@pytest.mark.parametrize("opts", [FP64, MIXED_TC], ids=["fp64", "mixed"])
def test_ragged_blocks_with_one_row_blocks(opts):
    """Blocks of 1, 2, 37, 1, 150 and 9 rows of a random diagonally dominant
    matrix: G^ element by element and the solve."""
    P = W.small_random_dd(200, 1, k_off=4, dd=1.5, seed=7)
    P.block_ptr = np.array([0, 1, 3, 40, 41, 191, 200], dtype=np.int64)
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr)
    S = make_solver(P, **opts)
    assert np.array_equal(S.interface(), o.c)
    bound = 1e-11 if opts is FP64 else 6e-4
    for b, ob in enumerate(o.blk):
        q0, q1, cols = S.ghat_layout(b)
        if (q1 - q0) * len(cols):
            scale = max(np.max(np.abs(ob["Ghat"])), 1e-300)
            assert np.max(np.abs(S.ghat_block(b) - ob["Ghat"])) <= bound * scale, b
    S.close()
    _check_solve(P, opts)


def test_tiny_and_identity_systems():
    """n = 2 with two one-row blocks (c = both rows), and A = I in 3 blocks
    (no coupling: x = f at once)."""
    A2 = np.array([[4.0, -1.0], [-2.0, 5.0]])
    _check_solve(_problem(A2, [0, 1, 2]), FP64, max_outer=0.5)
    I = sp.identity(50, format="csr")
    S, info = _check_solve(_problem(I, [0, 20, 21, 50], seed=2), FP64, max_outer=0.5)
    assert S.m == 0
    S.close()


def test_batch_mixing_degenerate_systems():
    """One handle with a single-block system, a system with one-row blocks and
    a slab system, and a zero right-hand side for one of them."""
    probs = [W.small_random_band(300, 1, 30, seed=8),
             W.small_convdiff_2d(10, 10),
             W.small_convdiff_3d(8, [2, 3, 3])]
    S = Solver.from_systems([(p.rowptr, p.colind, p.values, p.block_ptr) for p in probs],
                            tol_out=1e-12, tol_in=1e-8, **FP64)
    S.factor(dev(S.values_host))
    fs = [p.f.copy() for p in probs]
    fs[1][:] = 0.0
    x, info = S.solve(dev(np.concatenate(fs)))
    assert info["status"] == "DDPS_OK"
    x = host(x)
    for k, p in enumerate(probs):
        xk = x[S.sys_row_ptr[k]:S.sys_row_ptr[k + 1]]
        A = DDPSOracle(p.n, p.rowptr, p.colind, p.values, p.block_ptr, spikes=False).A
        if k == 1:
            assert np.all(xk == 0.0)
        else:
            assert relerr(xk, np.linalg.solve(A.toarray(), fs[k])) <= 1e-9, k
    S.close()


def test_direct_chain_with_a_one_sided_coupling():
    """A chain where column dropping removes the coupling of one block to its
    predecessor (an S_b with no correction): the direct reduced solve still
    solves G^ exactly (to FP32)."""
    P = W.small_convdiff_3d(10, [3, 4, 3], b=(0.0, 0.0, 40.0))
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, drop=("column", 0.5))
    S = make_solver(P, ("column", 0.5), reduced_solver=N.DDPS_REDUCED_DIRECT, **FP64)
    g = np.random.default_rng(3).standard_normal(o.m)
    zo, _ = o.reduced_solve(g, mode="direct")
    assert relerr(host(S.reduced_solve(dev(g))), zo) <= 1e-4
    S.close()
