"""Direct solve of the reduced system (Fig. 3 step 6.3 "directly"; Sec. 3
direct mode) for chains of blocks, through the C ABI, against the oracle's
dense solve of the same G^ (``DDPSOracle.reduced_solve(mode="direct")``) and
against the oracle's whole solve.  The block LU of G^ runs in FP32, so a
reduced solve matches to FP32 accuracy; the FP64 outer iteration then
recovers the full solution, with no inner iterations."""

import numpy as np
import pytest

import workloads as W
from gpu_helpers import dev, host, make_solver, relerr
from oracle.ddps_oracle import DDPSOracle
from paper_1008_1700_gb300 import Solver, native as N

pytestmark = pytest.mark.gpu

FP64_DIRECT = dict(factor_prec=N.DDPS_FP64, spike_prec=N.DDPS_FP64, ghat_prec=N.DDPS_FP64,
                   inner_prec=N.DDPS_FP64, reduced_solver=N.DDPS_REDUCED_DIRECT)
# the benched mixed form (FP32 factors, tensor-core spikes and LU updates, FP16 G^)
MIXED_DIRECT = dict(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_BF16X3, ghat_prec=N.DDPS_FP16,
                    inner_prec=N.DDPS_FP32, update_prec=N.DDPS_BF16X3,
                    reduced_solver=N.DDPS_REDUCED_DIRECT)

CHAINS = {
    "cd2d_24_p3": lambda: W.small_convdiff_2d(24, 3),
    "cd2d_cfg1": lambda: W.cfg1(),
    "cd3d_12_slabs": lambda: W.small_convdiff_3d(12, [3, 5, 4]),
    # 45 x 45 planes (2,025 rows per interface: 32 Gauss-Jordan steps, the last one
    # 41 columns wide, and ragged 128 x 128 GEMM tiles)
    "cd3d_45_slabs9": lambda: W.small_convdiff_3d(45, [5] * 9),
}


@pytest.fixture(scope="module", params=sorted(CHAINS))
def chain(request):
    P = CHAINS[request.param]()
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr,
                   spikes=request.param != "cd3d_45_slabs9")
    return request.param, P, o


def test_reduced_solve_matches_dense_solve(chain):
    name, P, o = chain
    if name == "cd3d_45_slabs9":
        pytest.skip("oracle G^ not formed for this size (full solve checked below)")
    S = make_solver(P, **FP64_DIRECT)
    for seed in (1, 2):
        g = np.random.default_rng(seed).standard_normal(o.m)
        z = host(S.reduced_solve(dev(g)))
        zo, _ = o.reduced_solve(g, mode="direct")
        # FP32 block LU of a G^ whose condition number is modest (M-matrices)
        assert relerr(z, zo) <= 1e-4, (name, seed)
    S.close()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_full_solve_with_direct_reduced_solve(chain, form):
    name, P, o = chain
    opts = FP64_DIRECT if form == "fp64" else MIXED_DIRECT
    S = make_solver(P, tol_out=1e-12, **opts)
    x, info = S.solve(dev(P.f))
    assert info["status"] == "DDPS_OK", info
    assert info["inner_iterations"] == 0
    x = host(x)
    assert np.max(np.abs(P.f - o.A @ x)) / np.max(np.abs(P.f)) <= 1e-12
    xo = np.linalg.solve(o.A.toarray(), P.f) if P.n <= 5000 else P.x_true
    assert relerr(x, xo) <= 1e-8, name
    S.close()


def test_direct_precond_is_the_exact_preconditioner_to_fp32():
    """Fig. 3 with the direct reduced solve equals the oracle's P^-1 y (direct
    mode) to FP32 accuracy, so the outer iteration needs at most 1.5 steps."""
    P = W.small_convdiff_3d(12, [3, 5, 4])
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr)
    S = make_solver(P, **FP64_DIRECT)
    y = np.random.default_rng(3).standard_normal(P.n)
    z = host(S.precond_apply(dev(y)))
    zo, _ = o.precond(y, mode="direct")
    assert relerr(z, zo) <= 1e-4
    x, info = S.solve(dev(P.f))
    assert info["outer_iterations"] <= 1.5


def test_direct_on_a_batch_of_chains():
    """Systems of different sizes stacked in one handle: one block LU per
    system, all systems' chain steps in the same launches."""
    probs = [W.small_convdiff_2d(N_, 8, seed=k) for k, N_ in enumerate([40, 33, 57, 24])]
    S = Solver.from_systems([(p.rowptr, p.colind, p.values, p.block_ptr) for p in probs],
                            tol_out=1e-12, **MIXED_DIRECT)
    S.factor(dev(S.values_host))
    x, info = S.solve(dev(np.concatenate([p.f for p in probs])))
    assert info["status"] == "DDPS_OK" and info["inner_iterations"] == 0
    x = host(x)
    for k, p in enumerate(probs):
        o = DDPSOracle(p.n, p.rowptr, p.colind, p.values, p.block_ptr, spikes=False)
        xo = np.linalg.solve(o.A.toarray(), p.f)
        assert relerr(x[S.sys_row_ptr[k]:S.sys_row_ptr[k + 1]], xo) <= 1e-8, k
    S.close()


def test_direct_rejects_partitions_that_are_not_chains():
    P = W.small_random_dd(301, 7, seed=9)  # random couplings between any blocks
    with pytest.raises(N.DDPSError, match="INVALID_ARG.*chain"):
        Solver(P.rowptr, P.colind, P.block_ptr, **FP64_DIRECT)
    Q = W.small_convdiff_2d(24, 3)
    with pytest.raises(N.DDPSError, match="INVALID_ARG.*EXPLICIT"):
        Solver(Q.rowptr, Q.colind, Q.block_ptr, ghat_mode=N.DDPS_GHAT_IMPLICIT,
               **{k: v for k, v in FP64_DIRECT.items()})
