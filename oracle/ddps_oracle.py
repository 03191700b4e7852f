"""Plain FP64 CPU oracle of DDPS (Manguoglu, "A domain-decomposing parallel
sparse linear system solver", arXiv 1008.1700).

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA solver.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it.  It shares no code with the CUDA path: it reads the same seeded
inputs (package ``workloads``) and nothing else.

It follows the paper's steps in the paper's order and notation, slowly and
without blocking or fusion:

* Fig. 2 step 1 / Eq. (1)-(2): ``A = D + R`` by block rows   -> ``split_block_rows``
* Fig. 2 step 2: exact LU of every ``A_ii``                    -> ``factor_blocks``
  (the paper calls a sparse direct solver, Pardiso, for this step; the oracle
  calls SuperLU through ``scipy.sparse.linalg.splu`` as that library step),
  or the approximate variant of Sec. 3, ILU(0) in the block's order -> ``ILU0``
* Fig. 2 step 3 / Sec. 3 dropping rule: ``R -> R~``           -> ``drop_columns``,
  plus the element-wise absolute rule of the random-band workload -> ``drop_entries``
* Fig. 2 step 5: ``c`` = nonzero columns of ``G``             -> ``interface_columns``
* Fig. 2 step 4: ``G = D~^-1 R~``, one column at a time        -> ``DDPSOracle`` spikes
* Fig. 3 steps 6.1-6.5: the preconditioner solve ``P z = y``   -> ``DDPSOracle.precond``
* Fig. 2 step 6 / Sec. 4 settings: outer BiCGStab (Templates book), stopping on
  ``||f - A x||_inf / ||f||_inf``, inner unpreconditioned BiCGStab on the reduced
  system with tolerance eps_in                                  -> ``bicgstab``

Readings taken where the paper is silent (also listed in the design notes):
the outer method is right-preconditioned BiCGStab with a convergence check at
both half steps (iteration counts ending in .5); the inner stopping test is
``||g^ - G^ z^||_2 <= eps_in ||g^||_2`` (relative to the right-hand side, so
that an initial guess can save iterations); the entry G(2, 9) of the worked
example is -0.004 as Eq. (6) prints it (Eq. (5) and Eq. (7) print +0.004; the
arithmetic of Eq. (4) gives -0.004).

Pins (tests in ``tests/test_oracle_pins.py``):
* every intermediate of the 9x9 worked example (Sec. 3, Eqs. (5)-(9)) to the
  printed digits;
* direct-mode exactness (Sec. 3: nothing dropped, exact LU, exact reduced
  solve => DDPS is a direct solver) against LAPACK dense LU on random systems;
* p = 1 (no coupling, c empty) reduces to one plain LU solve;
* the Krylov loop against closed forms (diagonal systems, 1 iteration) and the
  true-residual invariant on every workload family;
* Fig. 3 retrieval ``z = g - G z`` against the equivalent ``z = D~^-1 (y - R~ z^)``;
* ILU(0): (L U)_ij = a_ij on the block's pattern (the zero-fill identity),
  exact on patterns closed under elimination (a band with its full band),
  and brute-force elimination with the drop rule on tiny dense cases.
Parity unpinned: none of the functions above; the iteration *counts* of the
inexact (dropping / eps_in) variants have no independent reference and are
compared only through the true-residual invariant.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ----------------------------------------------------------------------------
# Fig. 2, step 1: A = D + R (Eq. (1)-(2))
# ----------------------------------------------------------------------------

def csr(n, rowptr, colind, values) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(values, np.float64), np.asarray(colind, np.int64),
                          np.asarray(rowptr, np.int64)), shape=(n, n))


def split_block_rows(A: sp.csr_matrix, block_ptr):
    """Return the diagonal blocks A_ii (list, CSC) and R = A - D (CSR, n x n).

    D holds the p diagonal blocks of A for the block-row partition given by
    ``block_ptr`` (Eq. (2)); R keeps every other entry of A (Eq. (1))."""
    A = A.tocoo()
    bp = np.asarray(block_ptr, dtype=np.int64)
    blk_r = np.searchsorted(bp, A.row, side="right") - 1
    blk_c = np.searchsorted(bp, A.col, side="right") - 1
    in_d = blk_r == blk_c
    n = A.shape[0]
    D_blocks = []
    for i in range(len(bp) - 1):
        sel = in_d & (blk_r == i)
        r0, r1 = bp[i], bp[i + 1]
        D_blocks.append(sp.csc_matrix((A.data[sel], (A.row[sel] - r0, A.col[sel] - r0)),
                                      shape=(r1 - r0, r1 - r0)))
    R = sp.csr_matrix((A.data[~in_d], (A.row[~in_d], A.col[~in_d])), shape=(n, n))
    R.sort_indices()
    return D_blocks, R


# ----------------------------------------------------------------------------
# Fig. 2, step 2: L_i U_i = A_ii (exact)
# ----------------------------------------------------------------------------

def factor_blocks(D_blocks, permc_spec="COLAMD"):
    """Exact sparse LU of each diagonal block (the library step of Fig. 2 step 2).
    ``permc_spec`` is SuperLU's column ordering; it changes the fill (and so
    the time and memory) and the rounding, not the factored matrix."""
    return [spla.splu(Dii.tocsc(), permc_spec=permc_spec) for Dii in D_blocks]


class ILU0:
    """Incomplete LU with zero fill of one diagonal block, in the block's own
    row order (Sec. 3: the block factors may be approximate; the paper names
    incomplete LU as the approximate choice).  L is unit lower triangular and
    U upper triangular, both on the sparsity pattern of the block; the
    entries are those of Gaussian elimination (row by row, IKJ form) with
    every update that would fall outside the pattern left out:
        for i, for k < i with a_ik in the pattern:
            a_ik = a_ik / a_kk
            a_ij = a_ij - a_ik a_kj   for every j > k with a_ij and a_kj in the pattern.
    ``solve(b)`` returns (L U)^-1 b."""

    def __init__(self, Dii):
        A = sp.csr_matrix(Dii, dtype=np.float64)
        A.sort_indices()
        n = A.shape[0]
        rp, ci = A.indptr, A.indices
        a = A.data.copy()
        for i in range(n):
            cols = ci[rp[i]:rp[i + 1]]
            pos = {int(c): rp[i] + t for t, c in enumerate(cols)}
            for t in range(rp[i], rp[i + 1]):
                k = int(ci[t])
                if k >= i:
                    break
                dk = rp[k] + int(np.searchsorted(ci[rp[k]:rp[k + 1]], k))
                a[t] = a[t] / a[dk]
                for u in range(dk + 1, rp[k + 1]):
                    j = int(ci[u])
                    if j in pos:
                        a[pos[j]] -= a[t] * a[u]
        F = sp.csr_matrix((a, ci.copy(), rp.copy()), shape=(n, n))
        self.L = (sp.tril(F, k=-1) + sp.identity(n)).tocsr()
        self.U = sp.triu(F).tocsr()

    def solve(self, b):
        b = np.asarray(b, dtype=np.float64)
        y = spla.spsolve_triangular(self.L, b, lower=True, unit_diagonal=True)
        return spla.spsolve_triangular(self.U, y, lower=False)


def ilu0_blocks(D_blocks):
    """ILU(0) of each diagonal block (the approximate variant of Fig. 2 step 2)."""
    return [ILU0(Dii) for Dii in D_blocks]


# ----------------------------------------------------------------------------
# Fig. 2, step 3: R~ from R by dropping
# ----------------------------------------------------------------------------

def drop_columns(R: sp.csr_matrix, block_ptr, delta: float) -> sp.csr_matrix:
    """Sec. 3 dropping rule: in block row R_i, column k is not considered when
    ||R_i(:, k)||_inf <= delta * max_j ||R_i(:, j)||_inf."""
    R = R.tocoo()
    bp = np.asarray(block_ptr, dtype=np.int64)
    blk = np.searchsorted(bp, R.row, side="right") - 1
    keep = np.zeros(R.nnz, dtype=bool)
    for i in range(len(bp) - 1):
        sel = np.nonzero(blk == i)[0]
        if sel.size == 0:
            continue
        cols = R.col[sel]
        absv = np.abs(R.data[sel])
        ucols, inv = np.unique(cols, return_inverse=True)
        colmax = np.zeros(len(ucols))
        np.maximum.at(colmax, inv, absv)
        kept_col = ~(colmax <= delta * colmax.max())
        keep[sel] = kept_col[inv]
    out = sp.csr_matrix((R.data[keep], (R.row[keep], R.col[keep])), shape=R.shape)
    out.sort_indices()
    return out


def drop_entries(R: sp.csr_matrix, tau: float) -> sp.csr_matrix:
    """Element-wise absolute rule: entries with |r_ij| < tau are dropped."""
    R = R.tocoo()
    keep = np.abs(R.data) >= tau
    out = sp.csr_matrix((R.data[keep], (R.row[keep], R.col[keep])), shape=R.shape)
    out.sort_indices()
    return out


# ----------------------------------------------------------------------------
# Fig. 2, step 5: c = indices of the nonzero columns of G
# ----------------------------------------------------------------------------

def interface_columns(Rt: sp.csr_matrix) -> np.ndarray:
    """Column k of G = D~^-1 R~ is nonzero exactly when column k of R~ is
    (D~ is nonsingular), so c is the sorted set of R~'s stored columns."""
    return np.unique(Rt.indices).astype(np.int64)


# ----------------------------------------------------------------------------
# BiCGStab (Templates book, right preconditioning) — Sec. 4 solver settings
# ----------------------------------------------------------------------------

def _norm(v, kind):
    return float(np.max(np.abs(v))) if kind == "inf" else float(np.linalg.norm(v))


def bicgstab(matvec, b, x0=None, precond=None, tol=1e-10, maxit=1000, norm="inf",
             ref=None, true_residual=True):
    """Preconditioned BiCGStab with the preconditioner applied on the right.

    Stops when ||r|| <= tol * ref (``ref`` defaults to ||b||), checked after
    each half step.  With ``true_residual`` the recurrence residual only
    triggers the test: the residual b - A x is recomputed and must pass too;
    if it does not, it replaces the recurrence residual and the loop goes on.

    Returns (x, info) with info["iterations"] counting half steps as 0.5.
    """
    M = precond if precond is not None else (lambda v: v.copy())
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if ref is None:
        ref = _norm(b, norm)
    info = {"iterations": 0.0, "converged": False, "breakdown": False, "history": [],
            "matvecs": 0, "precond": 0}
    if ref == 0.0:
        info["converged"] = True
        return np.zeros_like(b), info
    r = b - matvec(x) if x0 is not None else b.copy()
    if x0 is not None:
        info["matvecs"] += 1
    rn = _norm(r, norm)
    info["history"].append(rn / ref)
    if rn <= tol * ref:
        info["converged"] = True
        return x, info
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho = float(rhat @ r)
        if rho == 0.0:
            info["breakdown"] = True
            break
        if it == 1:
            p = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        phat = M(p)
        info["precond"] += 1
        v = matvec(phat)
        info["matvecs"] += 1
        sigma = float(rhat @ v)
        if sigma == 0.0:
            info["breakdown"] = True
            break
        alpha = rho / sigma
        s = r - alpha * v
        sn = _norm(s, norm)
        if sn <= tol * ref:
            xh = x + alpha * phat
            if not true_residual:
                x = xh
                info["iterations"] = it - 0.5
                info["converged"] = True
                info["history"].append(sn / ref)
                return x, info
            rt = b - matvec(xh)
            info["matvecs"] += 1
            if _norm(rt, norm) <= tol * ref:
                info["iterations"] = it - 0.5
                info["converged"] = True
                info["history"].append(_norm(rt, norm) / ref)
                return xh, info
        shat = M(s)
        info["precond"] += 1
        t = matvec(shat)
        info["matvecs"] += 1
        tt = float(t @ t)
        omega = float(t @ s) / tt if tt != 0.0 else 0.0
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rho_old = rho
        rn = _norm(r, norm)
        info["history"].append(rn / ref)
        info["iterations"] = float(it)
        if rn <= tol * ref:
            if not true_residual:
                info["converged"] = True
                return x, info
            rt = b - matvec(x)
            info["matvecs"] += 1
            if _norm(rt, norm) <= tol * ref:
                info["converged"] = True
                return x, info
            r = rt  # residual replacement
        if omega == 0.0:
            info["breakdown"] = True
            break
    return x, info


# ----------------------------------------------------------------------------
# The DDPS preprocessing (Fig. 2 steps 1-5) and preconditioner (Fig. 3)
# ----------------------------------------------------------------------------

class DDPSOracle:
    """DDPS stages 1-5 on construction; ``precond`` is Fig. 3; ``solve`` is step 6.

    ``drop`` is None, ("column", delta) for the Sec. 3 rule, or ("abs", tau)
    for the element-wise rule.  ``keep_full_G`` keeps the full spike columns
    G_i = A_ii^-1 R~_i(:, c_i) (needed by the retrieval z = g - G z of step
    6.5); without it only the rows of G that lie in c are kept and the
    retrieval uses the equivalent z = D~^-1 (y - R~ z^).
    """

    def __init__(self, n, rowptr, colind, values, block_ptr, drop=None, keep_full_G=True,
                 spikes=True, permc_spec="COLAMD", factor="lu"):
        self.n = int(n)
        self.A = csr(n, rowptr, colind, values)
        self.block_ptr = np.asarray(block_ptr, dtype=np.int64)
        self.p = len(self.block_ptr) - 1
        # step 1
        self.D_blocks, self.R = split_block_rows(self.A, self.block_ptr)
        # step 2
        # step 2: exact LU, or ILU(0) for the approximate variant (Sec. 3)
        self.lu = (ilu0_blocks(self.D_blocks) if factor == "ilu0"
                   else factor_blocks(self.D_blocks, permc_spec))
        # step 3
        if drop is None:
            self.Rt = self.R
        elif drop[0] == "column":
            self.Rt = drop_columns(self.R, self.block_ptr, float(drop[1]))
        elif drop[0] == "abs":
            self.Rt = drop_entries(self.R, float(drop[1]))
        else:
            raise ValueError(f"unknown drop rule {drop!r}")
        # step 5 (c only depends on the pattern of R~)
        self.c = interface_columns(self.Rt)
        self.m = len(self.c)
        self.pos = -np.ones(self.n, dtype=np.int64)
        self.pos[self.c] = np.arange(self.m)
        self.Rt_c = self.Rt.tocsc()[:, self.c].tocsr()  # R~(:, c), n x |c|
        self.keep_full_G = keep_full_G
        # per block: coupling columns c_i and the rows of the block that lie in c
        self.blk = []
        for i in range(self.p):
            r0, r1 = int(self.block_ptr[i]), int(self.block_ptr[i + 1])
            Ri = self.Rt[r0:r1, :]
            ci = np.unique(Ri.indices).astype(np.int64)
            rows_c = self.c[(self.c >= r0) & (self.c < r1)] - r0
            q0 = int(np.searchsorted(self.c, r0))
            q1 = int(np.searchsorted(self.c, r1))
            self.blk.append({"r0": r0, "r1": r1, "c_i": ci, "pos_i": self.pos[ci],
                             "rows_c": rows_c, "q0": q0, "q1": q1, "G": None, "Ghat": None})
        if spikes:
            self.form_spikes()

    # -- step 4: G = D~^-1 R~, one column at a time ---------------------------
    def spike_column(self, i: int, k: int) -> np.ndarray:
        """G_i(:, k) = A_ii^-1 R~_i(:, k) for a global column k (dense, length n_i)."""
        b = self.blk[i]
        col = self.Rt[b["r0"]:b["r1"], :].tocsc()[:, [k]].toarray().ravel()
        return self.lu[i].solve(col)

    def form_spikes(self):
        for i, b in enumerate(self.blk):
            ni = b["r1"] - b["r0"]
            ci = b["c_i"]
            Ri = self.Rt[b["r0"]:b["r1"], :].tocsc()[:, ci]
            Gi = np.zeros((ni, len(ci)))
            for j in range(len(ci)):
                Gi[:, j] = self.lu[i].solve(Ri[:, [j]].toarray().ravel())
            b["Ghat"] = Gi[b["rows_c"], :].copy()  # G(c ∩ block i, c_i)
            b["G"] = Gi if self.keep_full_G else None

    # -- Fig. 3 pieces ---------------------------------------------------------
    def block_solve(self, y: np.ndarray) -> np.ndarray:
        """6.1: g = D~^-1 y, block by block."""
        g = np.empty_like(y, dtype=np.float64)
        for i, b in enumerate(self.blk):
            g[b["r0"]:b["r1"]] = self.lu[i].solve(np.asarray(y[b["r0"]:b["r1"]], np.float64))
        return g

    def reduced_matvec(self, v: np.ndarray) -> np.ndarray:
        """w = G^ v with G^ = I(c,c) + G(c,c) (6.2), block row by block row."""
        w = v.copy()
        for b in self.blk:
            if b["q1"] > b["q0"] and len(b["c_i"]):
                w[b["q0"]:b["q1"]] += b["Ghat"] @ v[b["pos_i"]]
        return w

    def reduced_dense(self) -> np.ndarray:
        Gh = np.eye(self.m)
        for b in self.blk:
            if b["q1"] > b["q0"] and len(b["c_i"]):
                Gh[b["q0"]:b["q1"], b["pos_i"]] += b["Ghat"]
        return Gh

    def reduced_solve(self, ghat, mode="iterative", eps_in=1e-4, maxit_in=100, z0=None):
        """6.3: solve G^ z^ = g^ directly (dense LU) or by unpreconditioned BiCGStab."""
        if self.m == 0:
            return np.zeros(0), {"iterations": 0.0, "converged": True}
        if mode == "direct":
            return np.linalg.solve(self.reduced_dense(), ghat), {"iterations": 0.0, "converged": True}
        return bicgstab(self.reduced_matvec, ghat, x0=z0, tol=eps_in, maxit=maxit_in,
                        norm="2", ref=float(np.linalg.norm(ghat)), true_residual=False)

    def precond(self, y, mode="iterative", eps_in=1e-4, maxit_in=100, z0=None,
                retrieval="paper"):
        """Fig. 3: P z = y with P = D~ + R~.  Returns (z, info)."""
        g = self.block_solve(y)                                  # 6.1
        ghat = g[self.c]                                         # 6.2
        zhat, info = self.reduced_solve(ghat, mode, eps_in, maxit_in, z0)  # 6.3
        info["zhat"] = zhat
        info["ghat"] = ghat
        # 6.4 puts z^ into z(c); as G's nonzero columns are c, the product G z
        # of 6.5 is G(:, c) z^, and 6.5 then overwrites every entry of z.
        if retrieval == "paper" and self.keep_full_G:
            z = g.copy()                                         # 6.5: z = g - G z
            for b in self.blk:
                if len(b["c_i"]):
                    z[b["r0"]:b["r1"]] -= b["G"] @ zhat[b["pos_i"]]
        else:
            z = self.block_solve(y - self.Rt_c @ zhat)           # z = D~^-1 (y - R~ z^)
        return z, info

    # -- step 6: outer Krylov ----------------------------------------------------
    def solve(self, f, tol=1e-10, maxit=1000, mode="iterative", eps_in=1e-4, maxit_in=100,
              guess=None, retrieval="paper"):
        """Outer right-preconditioned BiCGStab on A with the DDPS preconditioner.

        ``guess`` (optional) is an initial guess for the reduced unknowns of the
        first preconditioner application (the learned-guess hook); later
        applications start from zero."""
        inner = []
        state = {"first": True}

        def M(y):
            z0 = guess if (state["first"] and guess is not None) else None
            state["first"] = False
            z, info = self.precond(y, mode, eps_in, maxit_in, z0, retrieval)
            inner.append(info["iterations"])
            return z

        x, info = bicgstab(lambda v: self.A @ v, f, precond=M, tol=tol, maxit=maxit,
                           norm="inf", ref=float(np.max(np.abs(f))), true_residual=True)
        info["inner_iterations"] = inner
        info["relres_inf"] = float(np.max(np.abs(f - self.A @ x)) / max(np.max(np.abs(f)), 1e-300))
        return x, info


# ----------------------------------------------------------------------------
# The plain definition x = A^-1 f for strictly diagonally dominant systems too
# large for one sparse LU
# ----------------------------------------------------------------------------

def jacobi_solution(A: sp.csr_matrix, f, tol=1e-16, maxit=5000):
    """x = A^-1 f by Jacobi iteration x <- D^-1 (f - (A - D) x), with a
    certified bound.  For A strictly diagonally dominant by rows, the
    iteration matrix B = -D^-1 (A - D) has q = ||B||_inf < 1 and every step
    satisfies ||x - x_k||_inf <= q / (1 - q) ||x_k - x_(k-1)||_inf; the loop
    stops once that bound is at most tol * ||x_k||_inf.  Returns (x, bound)
    where bound is the certified ||x - x_k||_inf (exact arithmetic; FP64
    rounding adds about n_row * eps * ||x||_inf).  This is the textbook
    stationary method; DDPS reaches the same x = A^-1 f in its direct mode
    (Sec. 3), which is the definition both are compared against."""
    A = sp.csr_matrix(A)
    d = A.diagonal()
    off = (A - sp.diags(d)).tocsr()
    q = float(np.max(np.asarray(abs(off).sum(axis=1)).ravel() / np.abs(d)))
    if not q < 1.0:
        raise ValueError("jacobi_solution needs a strictly row-diagonally dominant matrix")
    f = np.asarray(f, dtype=np.float64)
    x = f / d
    bound = np.inf
    for _ in range(maxit):
        xn = (f - off @ x) / d
        bound = q / (1.0 - q) * float(np.max(np.abs(xn - x)))
        x = xn
        if bound <= tol * float(np.max(np.abs(x))):
            break
    return x, bound


def relres_inf(A: sp.csr_matrix, x, f) -> float:
    return float(np.max(np.abs(f - A @ x)) / np.max(np.abs(f)))
