"""Pins of the CPU oracle against values it does not produce itself: the
paper's worked example (Sec. 3), LAPACK dense solves (direct-mode exactness),
closed forms and hand-made cases.  CPU only."""

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from conftest import read_golden
from oracle.ddps_oracle import (DDPSOracle, bicgstab, drop_columns, drop_entries,
                                interface_columns, split_block_rows, csr)

TOL_PRINTED = 5e-5 + 1e-12


@pytest.fixture(scope="module")
def example():
    gold = read_golden("worked_example_9x9.txt")
    P = W.worked_example(gold["A"], gold["block_ptr"].astype(np.int64), gold["f"])
    return gold, P, DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr)


def test_worked_example_split_and_c(example):
    gold, P, o = example
    A = gold["A"]
    # Eq. (2): D is the three 3x3 diagonal blocks; R = A - D (Eq. (1))
    D = np.zeros_like(A)
    for b in range(3):
        D[3 * b:3 * b + 3, 3 * b:3 * b + 3] = A[3 * b:3 * b + 3, 3 * b:3 * b + 3]
    assert np.array_equal(o.R.toarray(), A - D)
    for b in range(3):
        assert np.array_equal(o.D_blocks[b].toarray(), A[3 * b:3 * b + 3, 3 * b:3 * b + 3])
    # text after Eq. (5): unknowns 1, 2, 5 and 9 form the reduced system
    assert list(o.c + 1) == [int(v) for v in gold["c_one_based"]]


def test_worked_example_spikes_and_g(example):
    gold, P, o = example
    IG = np.eye(9)
    for b in o.blk:
        IG[b["r0"]:b["r1"], b["c_i"]] += b["G"]
    assert np.max(np.abs(IG - gold["I_plus_G"])) <= TOL_PRINTED       # Eq. (5), left
    g = o.block_solve(np.ones(9))
    assert np.max(np.abs(g - gold["g"])) <= TOL_PRINTED                # Eq. (5), right


def test_worked_example_reduced_system(example):
    gold, P, o = example
    assert np.max(np.abs(o.reduced_dense() - gold["Ghat"])) <= TOL_PRINTED   # Eq. (6)
    z, info = o.precond(np.ones(9), mode="direct")
    assert np.max(np.abs(info["zhat"] - gold["zhat"])) <= TOL_PRINTED
    assert np.max(np.abs(z - gold["x"])) <= TOL_PRINTED                      # Eq. (7)
    z2, _ = o.precond(np.ones(9), mode="direct", retrieval="split")
    assert np.max(np.abs(z2 - gold["x"])) <= TOL_PRINTED


def test_worked_example_iterative_inner(example):
    gold, P, o = example
    x, info = o.solve(np.ones(9), tol=1e-12, eps_in=1e-13, maxit_in=50)
    assert info["converged"]
    assert np.max(np.abs(x - gold["x"])) <= TOL_PRINTED


def _dense(P):
    return csr(P.n, P.rowptr, P.colind, P.values).toarray()


SMALL = [
    lambda: W.small_random_dd(60, 1, seed=1),
    lambda: W.small_random_dd(60, 2, seed=2),
    lambda: W.small_random_dd(61, 3, seed=3),
    lambda: W.small_random_dd(64, 4, seed=4, symmetric_pattern=True),
    lambda: W.small_convdiff_2d(8, 3),
    lambda: W.small_convdiff_3d(5, [2, 1, 2]),
    lambda: W.small_random_band(300, 4, 20, seed=5),
]


@pytest.mark.parametrize("make", SMALL)
def test_direct_mode_is_exact(make):
    """Sec. 3: no dropping + exact LU + exact reduced solve => DDPS is a direct
    solver.  One application of Fig. 3 to f equals LAPACK's dense solve."""
    P = make()
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr)
    x_ref = np.linalg.solve(_dense(P), P.f)
    for retrieval in ("paper", "split"):
        z, _ = o.precond(P.f, mode="direct", retrieval=retrieval)
        assert np.linalg.norm(z - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
    x, info = o.solve(P.f, tol=1e-12, mode="direct")
    assert info["iterations"] <= 1.0
    assert np.linalg.norm(x - x_ref) <= 1e-11 * np.linalg.norm(x_ref)


def test_single_block_is_plain_lu():
    """p = 1: R = 0, c is empty and Fig. 3 is one LU solve."""
    P = W.small_random_dd(50, 1, seed=11)
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr)
    assert o.m == 0 and o.R.nnz == 0
    z, _ = o.precond(P.f)
    x_ref = np.linalg.solve(_dense(P), P.f)
    assert np.linalg.norm(z - x_ref) <= 1e-12 * np.linalg.norm(x_ref)


def test_spikes_against_dense_inverse():
    """Fig. 2 step 4: G = D^-1 R; rows of the dense inverse times R."""
    P = W.small_random_band(200, 4, 15, seed=6)
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr)
    A = _dense(P)
    D = np.zeros_like(A)
    bp = P.block_ptr
    for i in range(P.p):
        D[bp[i]:bp[i + 1], bp[i]:bp[i + 1]] = A[bp[i]:bp[i + 1], bp[i]:bp[i + 1]]
    G = np.linalg.inv(D) @ (A - D)
    nzc = np.nonzero(np.any(A - D != 0, axis=0))[0]
    assert np.array_equal(o.c, nzc)
    for b in o.blk:
        assert np.allclose(b["G"], G[b["r0"]:b["r1"]][:, b["c_i"]], rtol=0, atol=1e-12)
    Gh = np.eye(len(nzc)) + G[np.ix_(nzc, nzc)]
    assert np.allclose(o.reduced_dense(), Gh, rtol=0, atol=1e-12)


@pytest.mark.parametrize("make,drop", [
    (lambda: W.small_convdiff_3d(8, [3, 3, 2]), None),
    (lambda: W.small_random_band(600, 4, 40, seed=3), ("abs", 1e-4)),
])
def test_implicit_reduced_product_identity(make, drop):
    """The identity the implicit G^ variant applies: for v on c,
    (I + G(c,c)) v = v + (D~^-1 (R~ v))(c), with R~ the dropped coupling and
    the dense inverse of D standing in for the factors."""
    P = make()
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, drop=drop)
    A = _dense(P)
    D = np.zeros_like(A)
    bp = P.block_ptr
    for i in range(P.p):
        D[bp[i]:bp[i + 1], bp[i]:bp[i + 1]] = A[bp[i]:bp[i + 1], bp[i]:bp[i + 1]]
    Rt = o.Rt.toarray()
    v = np.random.default_rng(11).standard_normal(o.m)
    vfull = np.zeros(P.n)
    vfull[o.c] = v
    w = v + np.linalg.solve(D, Rt @ vfull)[o.c]
    assert np.linalg.norm(o.reduced_matvec(v) - w) <= 1e-12 * np.linalg.norm(w)


def test_retrieval_forms_agree_with_inexact_inner():
    """6.5 (z = g - G z) and z = D^-1 (y - R z^) agree for any z^."""
    P = W.small_convdiff_2d(12, 4)
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr)
    y = np.random.default_rng(0).standard_normal(P.n)
    z1, i1 = o.precond(y, eps_in=1e-2, retrieval="paper")
    z2, i2 = o.precond(y, eps_in=1e-2, retrieval="split")
    assert np.array_equal(i1["zhat"], i2["zhat"])
    assert np.linalg.norm(z1 - z2) <= 1e-12 * np.linalg.norm(z1)


def test_column_drop_rule_hand_case():
    """Sec. 3 rule on a hand-made R: block 0 columns have inf-norms 4, 2, 1."""
    A = np.zeros((6, 6))
    A[np.arange(6), np.arange(6)] = 10.0
    A[0, 3] = 4.0; A[1, 3] = -1.0     # column 3: norm 4
    A[2, 4] = -2.0                    # column 4: norm 2
    A[1, 5] = 1.0                     # column 5: norm 1
    A[4, 0] = 3.0                     # block 1: a single column 0, norm 3
    M = sp.csr_matrix(A)
    bp = np.array([0, 3, 6])
    _, R = split_block_rows(M, bp)
    keep = lambda d: sorted(set(zip(*drop_columns(R, bp, d).nonzero())))
    assert keep(0.0) == sorted(set(zip(*R.nonzero())))
    # delta = 0.5: drop columns with norm <= 2 in block 0; block 1's only column has the max
    assert keep(0.5) == [(0, 3), (1, 3), (4, 0)]
    # delta = 0.25: norm 1 <= 1 dropped, norm 2 kept
    assert keep(0.25) == [(0, 3), (1, 3), (2, 4), (4, 0)]
    # delta = 1: every column has norm <= the max, so everything is dropped
    assert drop_columns(R, bp, 1.0).nnz == 0
    assert list(interface_columns(drop_columns(R, bp, 0.5))) == [0, 3]


def test_entry_drop_rule_hand_case():
    R = sp.csr_matrix(np.array([[0, 1e-5, 0], [2e-4, 0, -5e-5], [0, -1e-4, 0]]))
    Rt = drop_entries(R, 1e-4)
    assert sorted(zip(*Rt.nonzero())) == [(1, 0), (2, 1)]


def test_bicgstab_closed_forms():
    # exact preconditioner: the first half step already solves the system (0.5 iterations)
    d = np.array([1.0, 2.0, 3.0, 4.0])
    b = np.array([1.0, -1.0, 2.0, 0.5])
    x, info = bicgstab(lambda v: d * v, b, precond=lambda v: v / d, tol=1e-14)
    assert info["iterations"] == 0.5 and np.allclose(x, b / d, rtol=1e-15)
    # zero right-hand side: x = 0 without iterating
    x, info = bicgstab(lambda v: d * v, np.zeros(4))
    assert info["converged"] and not np.any(x)
    # a multiple of the identity: alpha = 1/2 exactly, again half an iteration
    x, info = bicgstab(lambda v: 2.0 * v, b, tol=1e-15)
    assert info["iterations"] == 0.5 and np.array_equal(x, b / 2.0)


def test_bicgstab_matches_lapack():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((40, 40)) + 40 * np.eye(40)
    b = rng.standard_normal(40)
    x, info = bicgstab(lambda v: A @ v, b, tol=1e-13, norm="2")
    assert info["converged"]
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-11 * np.linalg.norm(x)


@pytest.mark.parametrize("make,drop", [
    (lambda: W.small_convdiff_2d(24, 4), None),
    (lambda: W.small_convdiff_3d(8, [3, 2, 3]), None),
    (lambda: W.small_random_band(2000, 4, 100, seed=3), ("abs", 1e-4)),
    (lambda: W.small_random_band(2000, 4, 100, seed=4), ("column", 0.5)),
    (lambda: W.small_random_dd(400, 5, seed=8), ("column", 0.9)),
])
def test_residual_invariant_every_family(make, drop):
    """||f - A x||_inf / ||f||_inf <= 1e-10 for the inexact variants too (Sec. 3 outer layer)."""
    P = make()
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, drop=drop)
    x, info = o.solve(P.f, tol=1e-10, eps_in=1e-4, maxit_in=100)
    A = _dense(P)
    rel = np.max(np.abs(P.f - A @ x)) / np.max(np.abs(P.f))
    assert info["converged"] and rel <= 1e-10
    assert np.max(np.abs(x - P.x_true)) <= 1e-10 * np.linalg.cond(A, np.inf) * np.max(np.abs(P.x_true))


def test_cfg1_direct_agrees_with_global_lu():
    P = W.cfg1()
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr)
    assert o.m == 384  # 3 interfaces x 2 grid lines x 64
    x, info = o.solve(P.f, tol=1e-12, eps_in=1e-13, maxit_in=300)
    import scipy.sparse.linalg as spla
    x_ref = spla.spsolve(o.A.tocsc(), P.f)
    assert info["iterations"] <= 1.0
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_jacobi_reference_against_lapack_and_its_bound():
    """jacobi_solution (the definition x = A^-1 f for strictly diagonally
    dominant A): converged, it equals the LAPACK solve; stopped early, its
    certified bound q/(1-q) ||x_k - x_(k-1)||_inf covers the true error."""
    from oracle.ddps_oracle import jacobi_solution
    P = W.small_random_band(400, 4, 30, seed=7)  # diagonal 1.2 x the off-diagonal row sum
    A = _dense(P)
    x_ref = np.linalg.solve(A, P.f)
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, spikes=False)
    x, bound = jacobi_solution(o.A, P.f)
    assert np.max(np.abs(x - x_ref)) <= 1e-13 * np.max(np.abs(x_ref))
    for tol in (1e-3, 1e-6):
        xk, bk = jacobi_solution(o.A, P.f, tol=tol)
        err = np.max(np.abs(xk - x_ref))
        assert err <= bk and bk <= tol * np.max(np.abs(xk))
        assert err > 1e-3 * bk  # the bound is not vacuous
    with pytest.raises(ValueError):
        jacobi_solution(o.A - 2.0 * sp.diags(o.A.diagonal()) * 0.8, P.f)


def _ilu_brute(Ad):
    """Dense Gaussian elimination with every update outside the pattern of
    Ad dropped (the definition of ILU(0)), tiny matrices only."""
    n = Ad.shape[0]
    pat = Ad != 0
    a = Ad.astype(float).copy()
    for k in range(n):
        for i in range(k + 1, n):
            if not pat[i, k]:
                continue
            a[i, k] /= a[k, k]
            for j in range(k + 1, n):
                if pat[i, j] and pat[k, j]:
                    a[i, j] -= a[i, k] * a[k, j]
    return np.tril(a, -1) + np.eye(n), np.triu(a)


def test_ilu0_zero_fill_identity_and_brute_force():
    """ILU(0): L U agrees with A on A's pattern; L and U equal brute-force
    elimination with the zero-fill rule (KIJ order: a different loop order of
    the same definition); a solve applies (L U)^-1."""
    from oracle.ddps_oracle import ILU0
    for seed in range(4):
        P = W.small_random_dd(40, 1, k_off=3, dd=1.3, seed=seed)
        Ad = _dense(P)
        f = ILU0(sp.csr_matrix(Ad))
        L, U = f.L.toarray(), f.U.toarray()
        pat = Ad != 0
        assert np.max(np.abs((L @ U - Ad)[pat])) <= 1e-12 * np.max(np.abs(Ad))
        assert np.all(L[~pat & ~np.eye(40, dtype=bool)] == 0) and np.all(U[~pat] == 0)
        Lb, Ub = _ilu_brute(Ad)
        assert np.max(np.abs(L - Lb)) <= 1e-12 and np.max(np.abs(U - Ub)) <= 1e-12 * np.max(np.abs(Ad))
        b = np.random.default_rng(seed).standard_normal(40)
        assert np.max(np.abs(L @ U @ f.solve(b) - b)) <= 1e-11 * np.max(np.abs(b))


def test_ilu0_is_exact_on_a_closed_pattern():
    """On a matrix with a full band (every fill entry of Gaussian elimination
    lies inside the band) ILU(0) is the exact LU: L U = A and the solve is
    A^-1 b (checked against LAPACK)."""
    from oracle.ddps_oracle import ILU0
    rng = np.random.default_rng(5)
    n, bw = 60, 4
    Ad = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - bw), min(n, i + bw + 1)):
            Ad[i, j] = rng.standard_normal()
        Ad[i, i] = 2 * bw + 2.0
    f = ILU0(sp.csr_matrix(Ad))
    assert np.max(np.abs(f.L.toarray() @ f.U.toarray() - Ad)) <= 1e-12 * np.max(np.abs(Ad))
    b = rng.standard_normal(n)
    assert np.max(np.abs(f.solve(b) - np.linalg.solve(Ad, b))) <= 1e-12 * np.max(np.abs(np.linalg.solve(Ad, b)))


def test_ilu_variant_still_converges_to_the_solution():
    """DDPS with ILU(0) block factors (Sec. 3: approximate LU) is no longer a
    direct solver, but the outer Krylov iteration still reaches the true
    residual tolerance and the LAPACK solution."""
    P = W.small_convdiff_3d(10, [3, 4, 3])
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, factor="ilu0")
    x, info = o.solve(P.f, tol=1e-12, eps_in=1e-6, maxit_in=200)
    assert info["converged"] and info["iterations"] > 1.0
    x_ref = np.linalg.solve(_dense(P), P.f)
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
