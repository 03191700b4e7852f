"""ILU(0) block factors (factor_kind ILU0; Sec. 3: the block factors of
Fig. 2 step 2 may be approximate) through the C ABI against the oracle's
ILU(0) (``DDPSOracle(factor="ilu0")``): block solves with L~ U~, the spikes
G^ element by element, and the whole solve, whose outer iteration still
reaches the solution of A x = f."""

import numpy as np
import pytest

import workloads as W
from gpu_helpers import dev, host, make_solver, relerr
from oracle.ddps_oracle import DDPSOracle
from paper_1008_1700_gb300 import Solver, native as N

pytestmark = pytest.mark.gpu

ILU64 = dict(factor_prec=N.DDPS_FP64, spike_prec=N.DDPS_FP64, ghat_prec=N.DDPS_FP64,
             inner_prec=N.DDPS_FP64, factor_kind=N.DDPS_FACTOR_ILU0)
ILU32 = dict(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_FP32, ghat_prec=N.DDPS_FP32,
             inner_prec=N.DDPS_FP32, factor_kind=N.DDPS_FACTOR_ILU0)

PROBLEMS = {
    "cd2d_24_p3": (lambda: W.small_convdiff_2d(24, 3), None),
    "cd3d_12_slabs": (lambda: W.small_convdiff_3d(12, [3, 5, 4]), None),
    "randdd_301_p7": (lambda: W.small_random_dd(301, 7, seed=9), None),
    "band_3000_abs": (lambda: W.small_random_band(3000, 5, 200, seed=2), ("abs", 1e-4)),
}


@pytest.fixture(scope="module", params=sorted(PROBLEMS))
def case(request):
    make, drop = PROBLEMS[request.param]
    P = make()
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, drop=drop, factor="ilu0")
    return request.param, P, drop, o


@pytest.mark.parametrize("form,bound", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_ilu_block_solve_and_spikes(case, form, bound):
    name, P, drop, o = case
    S = make_solver(P, drop, **(ILU64 if form == "fp64" else ILU32))
    y = np.random.default_rng(1).standard_normal(P.n)
    assert relerr(host(S.block_solve(dev(y))), o.block_solve(y)) <= bound, name
    assert np.array_equal(S.interface(), o.c)
    for b, ob in enumerate(o.blk):
        q0, q1, cols = S.ghat_layout(b)
        if (q1 - q0) * len(cols) == 0:
            continue
        scale = max(np.max(np.abs(ob["Ghat"])), 1e-300)
        assert np.max(np.abs(S.ghat_block(b) - ob["Ghat"])) <= 10 * bound * scale, (name, b)
    S.close()


@pytest.mark.parametrize("form", ["fp64", "fp32", "fp32_direct"])
def test_ilu_full_solve(case, form):
    name, P, drop, o = case
    opts = dict(ILU64 if form == "fp64" else ILU32)
    if form == "fp32_direct":
        if name.startswith(("randdd", "band")):
            pytest.skip("not a chain of blocks")
        opts["reduced_solver"] = N.DDPS_REDUCED_DIRECT
    S = make_solver(P, drop, tol_out=1e-12, tol_in=1e-6, maxit_in=200, **opts)
    x, info = S.solve(dev(P.f))
    assert info["status"] == "DDPS_OK", info
    x = host(x)
    assert np.max(np.abs(P.f - o.A @ x)) / np.max(np.abs(P.f)) <= 1e-12
    xo = np.linalg.solve(o.A.toarray(), P.f)
    assert relerr(x, xo) <= 1e-8, name
    S.close()


def test_ilu_outer_iterations_against_the_oracle():
    """Same approximate preconditioner on both sides: the outer iteration
    counts of the FP64 GPU solve and of the oracle agree to one step."""
    P = W.small_convdiff_3d(12, [3, 5, 4])
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, factor="ilu0")
    S = make_solver(P, tol_out=1e-12, tol_in=1e-8, maxit_in=200, **ILU64)
    _, info = S.solve(dev(P.f))
    _, oinfo = o.solve(P.f, tol=1e-12, eps_in=1e-8, maxit_in=200)
    assert info["outer_iterations"] > 1.0
    assert abs(info["outer_iterations"] - oinfo["iterations"]) <= 1.0


def test_ilu_rejects_a_missing_diagonal():
    P = W.small_convdiff_2d(8, 2)
    keep = np.ones(P.nnz, dtype=bool)
    keep[P.rowptr[5]:P.rowptr[6]] = np.arange(P.rowptr[5], P.rowptr[6]) != \
        P.rowptr[5] + int(np.nonzero(P.colind[P.rowptr[5]:P.rowptr[6]] == 5)[0][0])
    colind = P.colind[keep]
    counts = np.diff(P.rowptr) - np.add.reduceat(~keep, P.rowptr[:-1].astype(np.int64))
    rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    with pytest.raises(N.DDPSError, match="INVALID_ARG.*diagonal"):
        Solver(rowptr, colind, P.block_ptr, **ILU64)
