"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on
the same seeded inputs: the worked example of Sec. 3, every step of Fig. 3,
the spikes G^ element by element and the full solve, for FP64 and the
mixed-precision forms."""

import numpy as np
import pytest
import torch

import workloads as W
from conftest import read_golden
from gpu_helpers import dev, host, make_solver, relerr
from oracle.ddps_oracle import DDPSOracle
from paper_1008_1700_gb300 import native as N

pytestmark = pytest.mark.gpu

FP64 = dict(factor_prec=N.DDPS_FP64, spike_prec=N.DDPS_FP64, ghat_prec=N.DDPS_FP64,
            inner_prec=N.DDPS_FP64)
MIXED = dict(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_FP32, ghat_prec=N.DDPS_FP32,
             inner_prec=N.DDPS_FP32)
MIXED_BF16 = dict(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_FP32, ghat_prec=N.DDPS_BF16,
                  inner_prec=N.DDPS_FP32)
# spike products on the tensor cores (bf16 operands, fp32 accumulation)
TC3 = dict(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_BF16X3, ghat_prec=N.DDPS_FP32,
           inner_prec=N.DDPS_FP32)
TC1 = dict(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_BF16, ghat_prec=N.DDPS_BF16,
           inner_prec=N.DDPS_FP32)
# the same products without the fused front GEMMs (every front takes the two
# tile products of each sweep), and with both kinds of fronts in one depth
TC3_TILES = dict(TC3, fused_rows=-1)
TC3_MIXED = dict(TC3, fused_rows=24)
# G^ stored in FP16 (FP32 accumulation), and the whole benched form: FP16 G^
# with tensor-core spike products and tensor-core LU block updates
TC3_F16 = dict(TC3, ghat_prec=N.DDPS_FP16)
BENCH = dict(TC3_F16, update_prec=N.DDPS_BF16X3)
# the benched form in passes of 128 coupling columns: passes that leave fronts
# inactive (cleared rows, zero-row reads, skipped stages in the backward) and
# fronts without active children (no gather)
BENCH_PASSES = dict(BENCH, rhs_chunk=128)
FORMS = {"mixed": MIXED, "tc3": TC3, "tc1": TC1, "tc3_tiles": TC3_TILES, "tc3_mixed": TC3_MIXED,
         "tc3_f16": TC3_F16, "bench": BENCH, "bench_passes": BENCH_PASSES}
# G^ applied without storing it: v + (D~^-1 R~ v)(c) by block solves
IMPLICIT64 = dict(FP64, ghat_mode=N.DDPS_GHAT_IMPLICIT)
IMPLICIT = dict(MIXED, ghat_mode=N.DDPS_GHAT_IMPLICIT)
# block LU of large fronts in blocks of 256 pivots, each block's update of the
# rest of the front on the tensor cores (bf16 high part + remainder)
TCLU = dict(TC3, update_prec=N.DDPS_BF16X3)


def test_worked_example_on_gpu():
    gold = read_golden("worked_example_9x9.txt")
    P = W.worked_example(gold["A"], gold["block_ptr"].astype(np.int64), gold["f"])
    S = make_solver(P, tol_out=1e-14, tol_in=1e-14, maxit_in=20, **FP64)
    assert list(S.interface() + 1) == [1, 2, 5, 9]
    Gh = np.eye(4)
    for b in range(3):
        q0, q1, cols = S.ghat_layout(b)
        Gh[q0:q1][:, cols] += S.ghat_block(b)
    assert np.max(np.abs(Gh - gold["Ghat"])) <= 5e-5
    g = host(S.block_solve(dev(np.ones(9))))
    assert np.max(np.abs(g - gold["g"])) <= 5e-5
    x, info = S.solve(dev(np.ones(9)))
    assert info["status"] == "DDPS_OK" and info["outer_iterations"] <= 1.0
    assert np.max(np.abs(host(x) - gold["x"])) <= 5e-5


PROBLEMS = {
    "cd2d_24_p3": (lambda: W.small_convdiff_2d(24, 3), None),
    "cd2d_cfg1": (lambda: W.cfg1(), None),
    "cd3d_12_slabs": (lambda: W.small_convdiff_3d(12, [3, 5, 4]), None),
    "randdd_301_p7": (lambda: W.small_random_dd(301, 7, seed=9), None),
    "band_3000_abs": (lambda: W.small_random_band(3000, 5, 200, seed=2), ("abs", 1e-4)),
    "band_2500_col": (lambda: W.small_random_band(2500, 4, 150, seed=3), ("column", 0.6)),
}


@pytest.fixture(scope="module", params=sorted(PROBLEMS))
def case(request):
    make, drop = PROBLEMS[request.param]
    P = make()
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, drop=drop)
    return request.param, P, drop, o


def test_ghat_matches_oracle_elementwise(case):
    name, P, drop, o = case
    S = make_solver(P, drop, **FP64)
    assert np.array_equal(S.interface(), o.c)
    for b, ob in enumerate(o.blk):
        q0, q1, cols = S.ghat_layout(b)
        assert (q0, q1) == (ob["q0"], ob["q1"])
        assert np.array_equal(cols, ob["pos_i"])
        if (q1 - q0) * len(cols) == 0:
            continue
        Gg = S.ghat_block(b)
        scale = max(np.max(np.abs(ob["Ghat"])), 1e-300)
        assert np.max(np.abs(Gg - ob["Ghat"])) <= 1e-11 * scale, (name, b)


def test_block_solve_and_reduced_matvec(case):
    name, P, drop, o = case
    S = make_solver(P, drop, **FP64)
    y = np.random.default_rng(1).standard_normal(P.n)
    assert relerr(host(S.block_solve(dev(y))), o.block_solve(y)) <= 1e-12
    if o.m:
        v = np.random.default_rng(2).standard_normal(o.m)
        assert relerr(host(S.reduced_matvec(dev(v))), o.reduced_matvec(v)) <= 1e-12
    yt = dev(y)
    assert relerr(host(S.spmv(yt)), o.A @ y) <= 1e-14


def test_precond_apply_direct_mode(case):
    """With a tight inner tolerance Fig. 3 returns P^-1 y; both sides agree."""
    name, P, drop, o = case
    S = make_solver(P, drop, tol_in=1e-13, maxit_in=500, **FP64)
    y = np.random.default_rng(3).standard_normal(P.n)
    z = host(S.precond_apply(dev(y)))
    zo, _ = o.precond(y, mode="direct")
    assert relerr(z, zo) <= 1e-9


# FP16 storage rounds every entry to 11 significant bits (relative 2^-11 =
# 4.9e-4 of the entry, at most that of the block's largest entry)
@pytest.mark.parametrize("form,bound", [("mixed", 2e-6), ("tc3", 1e-4), ("tc1", 3e-2),
                                        ("tc3_tiles", 1e-4), ("tc3_mixed", 1e-4),
                                        ("tc3_f16", 6e-4), ("bench", 6e-4),
                                        ("bench_passes", 6e-4)])
def test_ghat_precision_forms(case, form, bound):
    """G^ formed with FP32 factors: SIMT FP32 products, bf16x3 and bf16 tensor-core
    products (fused front GEMMs, tile products, or both); each within its
    arithmetic's accuracy of the FP64 oracle."""
    name, P, drop, o = case
    S = make_solver(P, drop, **FORMS[form])
    for b, ob in enumerate(o.blk):
        q0, q1, cols = S.ghat_layout(b)
        if (q1 - q0) * len(cols) == 0:
            continue
        scale = max(np.max(np.abs(ob["Ghat"])), 1e-300)
        assert np.max(np.abs(S.ghat_block(b) - ob["Ghat"])) <= bound * scale, (name, b)


@pytest.mark.parametrize("form,bound", [("implicit64", 1e-12), ("implicit", 1e-5)])
def test_implicit_reduced_matvec(case, form, bound):
    """The implicit G^ product (one R~ product and one block solve) against the
    oracle's stored G^; no spikes are kept, so G^'s blocks cannot be read."""
    name, P, drop, o = case
    S = make_solver(P, drop, **{"implicit64": IMPLICIT64, "implicit": IMPLICIT}[form])
    if not o.m:
        return
    for seed in (2, 5):
        v = np.random.default_rng(seed).standard_normal(o.m)
        assert relerr(host(S.reduced_matvec(dev(v))), o.reduced_matvec(v)) <= bound, (name, seed)
    with pytest.raises(N.DDPSError, match="STATE"):
        S.ghat_block(0)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16", "tc3", "tc1", "implicit64",
                                  "implicit", "tc3_f16", "bench", "bench_passes"])
def test_full_solve_parity(case, prec):
    name, P, drop, o = case
    opts = {"fp64": FP64, "mixed": MIXED, "mixed_bf16": MIXED_BF16, "tc3": TC3, "tc1": TC1,
            "implicit64": IMPLICIT64, "implicit": IMPLICIT, "tc3_f16": TC3_F16,
            "bench": BENCH, "bench_passes": BENCH_PASSES}[prec]
    S = make_solver(P, drop, tol_out=1e-12, tol_in=1e-6, maxit_in=200, **opts)
    x, info = S.solve(dev(P.f))
    assert info["status"] == "DDPS_OK", info
    x = host(x)
    xo, oinfo = o.solve(P.f, tol=1e-12, eps_in=1e-6, maxit_in=200)
    A = o.A
    assert np.max(np.abs(P.f - A @ x)) / np.max(np.abs(P.f)) <= 1e-12
    assert info["relres_inf"] <= 1e-12
    assert relerr(x, xo) <= 1e-8


def test_solve_is_deterministic():
    P = W.small_convdiff_3d(12, [3, 5, 4])
    S = make_solver(P, tol_out=1e-10, **MIXED)
    f = dev(P.f)
    x1, _ = S.solve(f)
    x1 = host(x1).copy()
    x2, _ = S.solve(f)
    assert np.array_equal(x1, host(x2))


def test_solve_host_buffers():
    P = W.small_convdiff_2d(20, 4)
    S = make_solver(P, tol_out=1e-12, tol_in=1e-10, **FP64)
    x, info = S.solve_host(P.f)
    assert info["status"] == "DDPS_OK"
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr)
    xo, _ = o.solve(P.f, tol=1e-12, eps_in=1e-10)
    assert relerr(x, xo) <= 1e-9


def test_batched_equals_per_system():
    """Independent systems stacked in one handle give each system's own result."""
    from paper_1008_1700_gb300 import Solver
    probs = [W.small_convdiff_2d(N, 4, seed=k) for k, N in enumerate([16, 21, 32, 19])]
    S = Solver.from_systems([(p.rowptr, p.colind, p.values, p.block_ptr) for p in probs],
                            tol_out=1e-12, tol_in=1e-8, **MIXED)
    S.factor(dev(S.values_host))
    x, info = S.solve(dev(np.concatenate([p.f for p in probs])))
    assert info["status"] == "DDPS_OK"
    x = host(x)
    for k, p in enumerate(probs):
        xk = x[S.sys_row_ptr[k]:S.sys_row_ptr[k + 1]]
        o = DDPSOracle(p.n, p.rowptr, p.colind, p.values, p.block_ptr)
        xo, _ = o.solve(p.f, tol=1e-12, eps_in=1e-8)
        assert relerr(xk, xo) <= 1e-8, k
        assert np.max(np.abs(p.f - o.A @ xk)) / np.max(np.abs(p.f)) <= 1e-12


LARGE_FRONTS = {
    # separators of up to 339 pivots (roots) and fronts of up to 428 rows
    "band_3000_abs": (lambda: W.small_random_band(3000, 5, 200, seed=2), ("abs", 1e-4)),
    # up to 619 pivots and 1,107 rows: three blocks of 256 pivots per front
    "band_6000_abs": (lambda: W.small_random_band(6000, 3, 400, seed=4), ("abs", 1e-4)),
}


@pytest.mark.parametrize("name", sorted(LARGE_FRONTS))
def test_lu_tensor_core_block_updates(name):
    """Block LU with the tensor-core block updates (ragged blocks, tiles and
    K): the block solve stays within the bf16x3 arithmetic's accuracy of the
    FP64 oracle (products good to about 2^-16, amplified by the blocks'
    condition numbers), and the outer FP64 iteration recovers the full
    solution."""
    make, drop = LARGE_FRONTS[name]
    P = make()
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, drop=drop)
    S = make_solver(P, drop, tol_out=1e-12, tol_in=1e-6, maxit_in=200, **TCLU)
    y = np.random.default_rng(4).standard_normal(P.n)
    assert relerr(host(S.block_solve(dev(y))), o.block_solve(y)) <= 2e-3
    x, info = S.solve(dev(P.f))
    assert info["status"] == "DDPS_OK", info
    xo, _ = o.solve(P.f, tol=1e-12, eps_in=1e-6, maxit_in=200)
    assert relerr(host(x), xo) <= 1e-8
    assert np.max(np.abs(P.f - o.A @ host(x))) / np.max(np.abs(P.f)) <= 1e-12


@pytest.mark.parametrize("opts", [FP64, MIXED], ids=["fp64", "mixed"])
def test_block_solve_of_a_wide_batch(opts):
    """A batch whose depths hold more fronts than two per SM: the block solve
    takes one warp per front there; it matches the oracle system by system."""
    from paper_1008_1700_gb300 import Solver
    probs = [W.small_convdiff_2d(24, 8, seed=50 + k) for k in range(48)]
    S = Solver.from_systems([(p.rowptr, p.colind, p.values, p.block_ptr) for p in probs], **opts)
    S.factor(dev(S.values_host))
    y = np.random.default_rng(8).standard_normal(S.n)
    g = host(S.block_solve(dev(y)))
    bound = 1e-12 if opts is FP64 else 1e-5
    for k, p in enumerate(probs):
        a, b = S.sys_row_ptr[k], S.sys_row_ptr[k + 1]
        o = DDPSOracle(p.n, p.rowptr, p.colind, p.values, p.block_ptr, spikes=False)
        assert relerr(g[a:b], o.block_solve(y[a:b])) <= bound, k


def test_batched_implicit_equals_explicit():
    """A stacked batch with the implicit G^ converges to the same solutions as
    the oracle; its inner iteration counts stay within one of the explicit
    FP32 G^ (the same operator, rounded differently)."""
    from paper_1008_1700_gb300 import Solver
    probs = [W.small_convdiff_2d(N, 4, seed=k) for k, N in enumerate([16, 21, 32, 19])]
    systems = [(p.rowptr, p.colind, p.values, p.block_ptr) for p in probs]
    f = dev(np.concatenate([p.f for p in probs]))
    infos = {}
    for form, opts in (("explicit", MIXED), ("implicit", IMPLICIT)):
        S = Solver.from_systems(systems, tol_out=1e-12, tol_in=1e-8, **opts)
        S.factor(dev(S.values_host))
        x, infos[form] = S.solve(f)
        assert infos[form]["status"] == "DDPS_OK"
        x = host(x)
        for k, p in enumerate(probs):
            o = DDPSOracle(p.n, p.rowptr, p.colind, p.values, p.block_ptr)
            xo, _ = o.solve(p.f, tol=1e-12, eps_in=1e-8)
            assert relerr(x[S.sys_row_ptr[k]:S.sys_row_ptr[k + 1]], xo) <= 1e-8, (form, k)
    assert abs(infos["explicit"]["first_inner_iters"] - infos["implicit"]["first_inner_iters"]) <= 1


def test_singular_block_is_reported():
    P = W.small_convdiff_2d(10, 2)
    vals = P.values.copy()
    # zero the whole row 3 inside its diagonal block: A_11 becomes singular
    r0, r1 = P.rowptr[3], P.rowptr[4]
    vals[r0:r1] = 0.0
    S = make_solver(W.small_convdiff_2d(10, 2))
    with pytest.raises(N.DDPSError, match="SINGULAR_BLOCK"):
        S.factor(dev(vals))


def test_not_converged_is_reported():
    P = W.small_convdiff_2d(24, 6)
    S = make_solver(P, tol_out=1e-14, maxit_out=1, tol_in=1e-1, maxit_in=1)
    x, info = S.solve(dev(P.f))
    assert info["status"] == "DDPS_ERR_NOT_CONVERGED"
    assert info["relres_inf"] > 1e-14 and np.isfinite(info["relres_inf"])


def test_reduced_guess_exact_and_rejected():
    P = W.small_convdiff_2d(24, 3)
    S = make_solver(P, tol_out=1e-10, tol_in=1e-8, **FP64)
    x, info0 = S.solve(dev(P.f))
    zhat, ghat = S.reduced_solution()
    # the exact reduced solution as guess: the first inner solve needs no iteration
    S.set_reduced_guess(zhat)
    x1, info1 = S.solve(dev(P.f))
    assert info1["guess_used"] == 1 and info1["first_inner_iters"] < info0["first_inner_iters"]
    assert info1["status"] == "DDPS_OK"
    # a guess worse than zero is rejected and the solve still converges
    S.set_reduced_guess(zhat * -50.0)
    x2, info2 = S.solve(dev(P.f))
    assert info2["guess_used"] == 0 and info2["status"] == "DDPS_OK"
    S.set_reduced_guess(None)


def test_batch_every_system_meets_tolerance():
    """A batch shaped like the 256-system workload (grid sides 32..80, 8 grid-line
    blocks each): every system's recomputed residual meets tol_out, the reported
    worst residual agrees, and sampled systems match the oracle."""
    from paper_1008_1700_gb300 import Solver
    sides = np.random.default_rng(11).integers(32, 81, 12)
    probs = [W.small_convdiff_2d(int(N), 8, seed=1000 + k) for k, N in enumerate(sides)]
    S = Solver.from_systems([(p.rowptr, p.colind, p.values, p.block_ptr) for p in probs],
                            tol_out=1e-10, tol_in=1e-4, **TC3)
    S.factor(dev(S.values_host))
    x, info = S.solve(dev(np.concatenate([p.f for p in probs])))
    x = host(x)
    worst = 0.0
    for k, p in enumerate(probs):
        xk = x[S.sys_row_ptr[k]:S.sys_row_ptr[k + 1]]
        A = DDPSOracle(p.n, p.rowptr, p.colind, p.values, p.block_ptr, spikes=False).A
        rr = np.max(np.abs(p.f - A @ xk)) / np.max(np.abs(p.f))
        worst = max(worst, rr)
        assert rr <= 1e-10, (k, rr)
    assert info["status"] == "DDPS_OK" and info["converged"] == 1
    assert abs(info["relres_inf"] - worst) <= 1e-3 * worst + 1e-18
    for k in (0, 7):
        p = probs[k]
        xo, _ = DDPSOracle(p.n, p.rowptr, p.colind, p.values, p.block_ptr).solve(
            p.f, tol=1e-12, eps_in=1e-8)
        assert relerr(x[S.sys_row_ptr[k]:S.sys_row_ptr[k + 1]], xo) <= 1e-7


@pytest.mark.parametrize("fused_rows", [0, -1])
def test_bounded_wait_reports_timeout_and_context_survives(fused_rows):
    """Failure path of the tensor-core spike kernels (fused front GEMM, tile
    products): with debug_wait_timeout the kernel waits on an mbarrier that
    nothing arrives at; the bounded wait runs out, the kernel frees its tensor
    memory and returns, ddps_factor reports DDPS_ERR_TIMEOUT, and the context
    stays usable for a normal solve."""
    P = W.small_convdiff_2d(24, 3)
    from paper_1008_1700_gb300 import Solver
    S = Solver(P.rowptr, P.colind, P.block_ptr, debug_wait_timeout=1, fused_rows=fused_rows,
               **TC3)
    with pytest.raises(N.DDPSError, match="TIMEOUT"):
        S.factor(dev(P.values))
    S.close()
    S2 = make_solver(P, tol_out=1e-12, tol_in=1e-8, **TC3)
    x, info = S2.solve(dev(P.f))
    assert info["status"] == "DDPS_OK" and info["relres_inf"] <= 1e-12


def test_several_rhs_and_initial_guess():
    """ddps_solve with nrhs right-hand sides (one after the other with the same
    factors) and with initial guesses: each column matches the oracle; a guess
    equal to the solution returns at once; a zero right-hand side gives x = 0
    whatever the guess."""
    P = W.small_convdiff_3d(12, [3, 5, 4])
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr)
    S = make_solver(P, tol_out=1e-12, tol_in=1e-8, **MIXED)
    rng = np.random.default_rng(21)
    F = np.stack([P.f, rng.standard_normal(P.n), np.zeros(P.n)])
    X, info = S.solve(dev(F))
    assert info["status"] == "DDPS_OK"
    X = host(X)
    for j in range(2):
        xo, _ = o.solve(F[j], tol=1e-12, eps_in=1e-8)
        assert relerr(X[j], xo) <= 1e-8, j
    assert np.all(X[2] == 0.0)
    # the first column's solution as its guess: no iteration; a perturbed guess converges
    X0 = np.stack([X[0], X[1] + 1e-3 * rng.standard_normal(P.n), rng.standard_normal(P.n)])
    X2, info2 = S.solve(dev(F), x0=dev(X0))
    X2 = host(X2)
    assert info2["status"] == "DDPS_OK"
    assert np.array_equal(X2[0], X[0])
    assert relerr(X2[1], X[1]) <= 1e-9
    assert np.all(X2[2] == 0.0)
    # host buffers give the same as device buffers
    Xh, infoh = S.solve_host(F)
    assert infoh["status"] == "DDPS_OK" and np.array_equal(Xh, X)


def test_factor_from_host_values():
    """ddps_factor_host (values in host memory) factors exactly as ddps_factor."""
    P = W.small_random_band(3000, 5, 200, seed=2)
    S1 = make_solver(P, ("abs", 1e-4), **TCLU)
    S2 = make_solver(P, ("abs", 1e-4), **TCLU)
    S2.factor(np.asarray(P.values))
    y = dev(np.random.default_rng(5).standard_normal(P.n))
    assert np.array_equal(host(S1.block_solve(y)), host(S2.block_solve(y)))
    assert np.array_equal(S1.ghat_block(2), S2.ghat_block(2))


@pytest.mark.parametrize("form", ["fp64", "tc3", "implicit", "direct"])
def test_graph_replay_matches_plain_launches(form):
    """The factor phase, the inner iterations and (direct mode) the whole
    preconditioner are replayed from CUDA graphs after their first use; the
    results are bitwise those of plain launches, over repeated factor + solve
    calls, and with fewer host-side launches."""
    opts = {"fp64": FP64, "tc3": dict(TC3, update_prec=N.DDPS_BF16X3), "implicit": IMPLICIT,
            "direct": dict(TC3, reduced_solver=N.DDPS_REDUCED_DIRECT)}[form]
    probs = [W.small_convdiff_3d(12, [3, 5, 4]), W.small_convdiff_3d(10, [4, 3, 3], seed=3)]
    from paper_1008_1700_gb300 import Solver
    xs = {}
    for graphs in (0, 1):
        S = Solver.from_systems([(p.rowptr, p.colind, p.values, p.block_ptr) for p in probs],
                                tol_out=1e-12, tol_in=1e-6, use_graphs=graphs, **opts)
        f = dev(np.concatenate([p.f for p in probs]))
        out = []
        for rep in range(3):
            S.factor(dev(S.values_host * (1.0 + 0.01 * rep)))
            x, info = S.solve(f)
            assert info["status"] == "DDPS_OK"
            out.append(host(x).copy())
        xs[graphs] = out
        S.close()
    for rep in range(3):
        assert np.array_equal(xs[0][rep], xs[1][rep]), rep


@pytest.mark.parametrize("opts", [FP64, MIXED], ids=["fp64", "mixed"])
def test_persistent_sweeps_match_level_launches(opts):
    """The deep levels of small fronts swept by one persistent launch per
    sweep (fronts ordered by completion flags) give the block solves of one
    launch per depth (whose launch shapes, and so summation orders, the
    autotuner may choose differently), on a 3-D slab system and on a wide
    batch; both match the oracle's block solve to the arithmetic's accuracy."""
    from paper_1008_1700_gb300 import Solver
    cases = [[W.small_convdiff_3d(16, [5, 6, 5])],
             [W.small_convdiff_2d(24, 8, seed=60 + k) for k in range(40)]]
    for probs in cases:
        gs = []
        for persist in (0, 1):
            S = Solver.from_systems([(p.rowptr, p.colind, p.values, p.block_ptr) for p in probs],
                                    persistent_solve=persist, **opts)
            S.factor(dev(S.values_host))
            y = dev(np.random.default_rng(9).standard_normal(S.n))
            gs.append(host(S.block_solve(y)).copy())
            x, info = S.solve(dev(np.concatenate([p.f for p in probs])))
            assert info["status"] == "DDPS_OK"
            S.close()
        bound = 1e-12 if opts is FP64 else 1e-5
        assert relerr(gs[1], gs[0]) <= bound
        p = probs[0]
        o = DDPSOracle(p.n, p.rowptr, p.colind, p.values, p.block_ptr, spikes=False)
        y0 = np.random.default_rng(9).standard_normal(sum(q.n for q in probs))[:p.n]
        assert relerr(gs[1][:p.n], o.block_solve(y0)) <= (1e-12 if opts is FP64 else 1e-5)


def test_autotuned_block_solve_shapes(tmp_path, monkeypatch):
    """The first factor times every candidate launch shape of each block-solve
    depth and keeps the fastest; the choices are reported, cached in the JSON
    file DDPS_TUNE_CACHE names, and the tuned block solve matches the oracle
    like the fixed rules do."""
    import json
    monkeypatch.setenv("DDPS_TUNE_CACHE", str(tmp_path / "tune.json"))
    P = W.small_random_band(3000, 5, 200, seed=2)  # fronts of up to 428 rows: clusters compete
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, drop=("abs", 1e-4),
                   spikes=False)
    y = np.random.default_rng(4).standard_normal(P.n)
    for tune in (0, 1):
        S = make_solver(P, ("abs", 1e-4), autotune=tune, persistent_solve=0, **FP64)
        t = S.tuning()
        assert t["tuned"] == bool(tune)
        if tune:
            names = {"warp", "cta8", "cl1", "cl2", "cl4", "cl8"}
            assert t["levels"] and all(l["fwd"] in names and l["bwd"] in names for l in t["levels"])
        assert relerr(host(S.block_solve(dev(y))), o.block_solve(y)) <= 1e-12
        S.close()
    cache = json.loads((tmp_path / "tune.json").read_text())
    assert cache and all(v in range(6) for v in cache.values())


def test_csr_kernels_agree():
    """Every kernel of the products with A and R~ (row blocks, 4 or 8 lanes per
    row, row blocks with all loads issued at once, 32-row groups per warp)
    against A y; the row-block and row-group kernels sum in the same order
    with the same rounding, so they agree bit for bit, and a whole solve
    converges with each."""
    P = W.small_convdiff_2d(151, 5)  # 22,801 rows in ragged blocks, nnz not a multiple of 4
    A = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, spikes=False).A
    y = np.random.default_rng(5).standard_normal(P.n)
    out = {}
    for kernel in range(5):
        S = make_solver(P, csr_kernel=kernel, tol_out=1e-12, **FP64)
        assert S.tuning()["spmv"] == ["stream", "vec4", "vec8", "block", "warp"][kernel]
        out[kernel] = host(S.spmv(dev(y)))
        assert relerr(out[kernel], A @ y) <= 1e-14, kernel
        x, info = S.solve(dev(P.f))
        assert info["status"] == "DDPS_OK", (kernel, info)
        assert np.max(np.abs(P.f - A @ host(x))) / np.max(np.abs(P.f)) <= 1e-12, kernel
        S.close()
    assert P.colind.size % 4 != 0
    assert np.array_equal(out[0], out[3]) and np.array_equal(out[0], out[4])
    with pytest.raises(N.DDPSError, match="csr_kernel"):
        make_solver(P, csr_kernel=5, **FP64)
