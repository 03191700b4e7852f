"""Seeded generators for the synthetic workloads.

Every matrix is returned in CSR form (int32 row pointers and column indices,
float64 values, columns sorted inside each row, no stored zeros) together with
a block-row partition ``block_ptr`` (int64, p+1 entries) and a right-hand side.

Workload recipe (all randomness from numpy's PCG64 through ``default_rng``):

* 2-D / 3-D convection-diffusion: ``-Lap(u) + b . grad(u)`` on the unit square
  or cube, homogeneous Dirichlet boundary, N interior points per side,
  h = 1/(N+1), second-order central differences, the whole row scaled by h^2.
  Diagonal 2d; the neighbour at -h along axis k gets ``-1 - b_k h/2`` and the
  one at +h gets ``-1 + b_k h/2``.  Natural ordering, x fastest.
* random band: per row, ``k_off`` distinct off-diagonal columns; each is
  long-range (uniform over [0, n)) with probability ``p_long``, otherwise
  uniform in [i - hw, i + hw]; picks that fall outside [0, n), on the diagonal
  or on a column already taken are redrawn.  Off-diagonal values ~ N(0, 1);
  the diagonal is ``dd`` times the off-diagonal absolute row sum.
* right-hand side: ``f = A x_true`` with ``x_true ~ U[-1, 1]`` unless stated.

The five named workloads (``cfg1`` .. ``cfg5``) fix the sizes, coefficients and
seeds; the ``small_*`` helpers give the same families at test sizes.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One linear system ``A x = f`` with a block-row partition."""

    n: int
    rowptr: np.ndarray  # int32 [n+1]
    colind: np.ndarray  # int32 [nnz]
    values: np.ndarray  # float64 [nnz]
    block_ptr: np.ndarray  # int64 [p+1]
    f: np.ndarray  # float64 [n]
    x_true: np.ndarray | None = None  # float64 [n] when f = A x_true
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def p(self) -> int:
        return len(self.block_ptr) - 1


# ----------------------------------------------------------------------------
# CSR assembly helpers (input construction only)
# ----------------------------------------------------------------------------

def _coo_to_csr(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    vals = vals[order]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit in int32")
    return rowptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64)


def _rhs_from_solution(rowptr, colind, values, x):
    """f_i = sum_j a_ij x_j, summed row by row (builds the input right-hand side)."""
    prod = values * x[colind]
    n = len(rowptr) - 1
    f = np.zeros(n)
    nz_rows = np.diff(rowptr) > 0
    f[nz_rows] = np.add.reduceat(prod, rowptr[:-1][nz_rows].astype(np.int64))
    return f


# ----------------------------------------------------------------------------
# Matrix families
# ----------------------------------------------------------------------------

def convdiff_2d(N: int, bx: float, by: float):
    """5-point convection-diffusion on an N x N interior grid (scaled by h^2)."""
    h = 1.0 / (N + 1)
    n = N * N
    idx = np.arange(n, dtype=np.int64)
    x = idx % N
    y = idx // N
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 4.0)]
    for (dx, dy, b) in ((-1, 0, bx), (1, 0, bx), (0, -1, by), (0, 1, by)):
        ok = (x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N)
        s = dx + dy  # -1 for the lower neighbour, +1 for the upper one
        v = -1.0 + s * b * h / 2.0
        rows.append(idx[ok])
        cols.append(idx[ok] + dx + dy * N)
        vals.append(np.full(int(ok.sum()), v))
    return _coo_to_csr(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def convdiff_3d(N: int, bx: float, by: float, bz: float):
    """7-point convection-diffusion on an N^3 interior grid (scaled by h^2)."""
    h = 1.0 / (N + 1)
    n = N * N * N
    idx = np.arange(n, dtype=np.int64)
    x = idx % N
    y = (idx // N) % N
    z = idx // (N * N)
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 6.0)]
    for (dx, dy, dz, b) in ((-1, 0, 0, bx), (1, 0, 0, bx), (0, -1, 0, by), (0, 1, 0, by),
                            (0, 0, -1, bz), (0, 0, 1, bz)):
        ok = ((x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N)
              & (z + dz >= 0) & (z + dz < N))
        s = dx + dy + dz
        v = -1.0 + s * b * h / 2.0
        rows.append(idx[ok])
        cols.append(idx[ok] + dx + dy * N + dz * N * N)
        vals.append(np.full(int(ok.sum()), v))
    return _coo_to_csr(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def random_band(n: int, hw: int, k_off: int, p_long: float, dd: float, rng):
    """Random nonsymmetric band matrix with a few long-range entries."""
    rows = np.repeat(np.arange(n, dtype=np.int64), k_off)
    cols = np.empty(n * k_off, dtype=np.int64)
    need = np.ones(n * k_off, dtype=bool)
    for _ in range(200):
        m = int(need.sum())
        if m == 0:
            break
        r = rows[need]
        longr = rng.random(m) < p_long
        cand = np.where(longr, rng.integers(0, n, m), r + rng.integers(-hw, hw + 1, m))
        cols[need] = cand
        bad = (cols < 0) | (cols >= n) | (cols == rows)
        # duplicates inside a row: keep the first occurrence, redraw the rest
        c2 = np.where(bad, -1 - np.arange(n * k_off), cols)  # unique sentinels for bad slots
        key = rows * (2 * n + 2) + c2
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup_sorted = np.zeros(len(ks), dtype=bool)
        dup_sorted[1:] = ks[1:] == ks[:-1]
        dup = np.zeros(len(ks), dtype=bool)
        dup[order] = dup_sorted
        need = bad | dup
    else:
        raise RuntimeError("random_band: could not place all entries")
    offv = rng.standard_normal(n * k_off)
    absum = np.bincount(rows, weights=np.abs(offv), minlength=n)
    diag = dd * absum
    allr = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    allc = np.concatenate([cols, np.arange(n, dtype=np.int64)])
    allv = np.concatenate([offv, diag])
    return _coo_to_csr(n, allr, allc, allv)


def random_dd(n: int, k_off: int, dd: float, rng, symmetric_pattern: bool = False):
    """Small random sparse matrix, strictly diagonally dominant by factor ``dd``."""
    rows = np.repeat(np.arange(n, dtype=np.int64), k_off)
    cols = rng.integers(0, n, n * k_off)
    keep = cols != rows
    rows, cols = rows[keep], cols[keep]
    if symmetric_pattern:
        rows, cols = np.concatenate([rows, cols]), np.concatenate([cols, rows])
    key = np.unique(rows * n + cols)
    rows, cols = key // n, key % n
    offv = rng.standard_normal(len(rows))
    absum = np.bincount(rows, weights=np.abs(offv), minlength=n)
    diag = dd * absum + 1.0
    allr = np.concatenate([rows, np.arange(n)])
    allc = np.concatenate([cols, np.arange(n)])
    allv = np.concatenate([offv, diag])
    return _coo_to_csr(n, allr, allc, allv)


# ----------------------------------------------------------------------------
# Partitions
# ----------------------------------------------------------------------------

def equal_blocks(n: int, p: int) -> np.ndarray:
    """Block boundaries floor(i n / p)."""
    return np.array([(i * n) // p for i in range(p + 1)], dtype=np.int64)


def grid_line_blocks(N: int, p: int) -> np.ndarray:
    """Split the N grid lines of a 2-D grid into p groups of floor/ceil(N/p) lines."""
    sizes = [N // p + (1 if i < N % p else 0) for i in range(p)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64) * N


def slab_blocks(N: int, planes: list[int]) -> np.ndarray:
    """z-slab partition of an N^3 grid; ``planes`` lists each slab's plane count."""
    if sum(planes) != N:
        raise ValueError("slab plane counts must sum to N")
    return np.concatenate([[0], np.cumsum(planes)]).astype(np.int64) * (N * N)


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

def _xtrue(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def _problem(n, csr, block_ptr, x_true, name, meta, f=None):
    rowptr, colind, values = csr
    if f is None:
        f = _rhs_from_solution(rowptr, colind, values, x_true)
    return Problem(n=n, rowptr=rowptr, colind=colind, values=values, block_ptr=block_ptr,
                   f=f, x_true=x_true, name=name, meta=meta)


def cfg1() -> Problem:
    """2-D convection-diffusion, 64 x 64, b = (10, 10), 4 equal block rows, no dropping."""
    N = 64
    n = N * N
    return _problem(n, convdiff_2d(N, 10.0, 10.0), equal_blocks(n, 4), _xtrue(n, 0),
                    "cfg1_cd2d_64_p4", {"N": N, "b": (10.0, 10.0)})


def cfg2_slab_planes() -> list[int]:
    """16 z-slabs of 3..5 planes summing to 64: 16 x 4, then four seeded +-1 moves."""
    sizes = [4] * 16
    rng = np.random.default_rng(0)
    moves = 0
    while moves < 4:
        i, j = (int(v) for v in rng.integers(0, 16, 2))
        if i != j and sizes[i] < 5 and sizes[j] > 3:
            sizes[i] += 1
            sizes[j] -= 1
            moves += 1
    return sizes


def cfg2() -> Problem:
    """3-D convection-diffusion, 64^3, one convection constant per axis ~ U[0, 50]."""
    N = 64
    n = N ** 3
    b = np.random.default_rng([0, 1]).uniform(0.0, 50.0, 3)
    planes = cfg2_slab_planes()
    return _problem(n, convdiff_3d(N, *b), slab_blocks(N, planes), _xtrue(n, 0),
                    "cfg2_cd3d_64_slabs16", {"N": N, "b": tuple(float(v) for v in b),
                                             "planes": planes})


def cfg3_sides(count: int = 256) -> np.ndarray:
    return np.random.default_rng(3).integers(32, 129, count)


def cfg3(count: int = 256) -> list[Problem]:
    """``count`` independent 2-D convection-diffusion systems, side ~ U{32..128}, 8 blocks each."""
    out = []
    for k, N in enumerate(cfg3_sides(count)):
        N = int(N)
        n = N * N
        out.append(_problem(n, convdiff_2d(N, 10.0, 10.0), grid_line_blocks(N, 8),
                            _xtrue(n, 1000 + k), f"cfg3_sys{k}_N{N}", {"N": N, "b": (10.0, 10.0)}))
    return out


def cfg4(n: int = 1_000_000, p: int = 128) -> Problem:
    """Random nonsymmetric band (half-width 2000, 11 off-diagonals per row, 1% long range)."""
    rng = np.random.default_rng([0, 4])
    csr = random_band(n, 2000, 11, 0.01, 1.2, rng)
    return _problem(n, csr, equal_blocks(n, p), _xtrue(n, 0), f"cfg4_randband_{n}_p{p}",
                    {"hw": 2000, "k_off": 11, "p_long": 0.01, "dd": 1.2, "drop_abs": 1e-4})


def cfg5_coeff(t: int) -> float:
    """Convection coefficient of time step t (1-based): 20 + 10 sin(2 pi t / 200)."""
    return 20.0 + 10.0 * math.sin(2.0 * math.pi * t / 200.0)


def cfg5(t: int, N: int = 48, slabs: int = 8) -> Problem:
    """Time step t of the 3-D 48^3 sequence: fixed source f = h^2, 8 slabs of 6 planes."""
    b = cfg5_coeff(t)
    n = N ** 3
    h = 1.0 / (N + 1)
    planes = [N // slabs + (1 if i < N % slabs else 0) for i in range(slabs)]
    csr = convdiff_3d(N, b, b, b)
    return _problem(n, csr, slab_blocks(N, planes), None, f"cfg5_cd3d_{N}_t{t}",
                    {"N": N, "t": t, "b": b}, f=np.full(n, h * h))


# ----------------------------------------------------------------------------
# Small members of the same families (test sizes)
# ----------------------------------------------------------------------------

def small_convdiff_2d(N: int, p: int, b=(10.0, 10.0), seed: int = 0) -> Problem:
    n = N * N
    return _problem(n, convdiff_2d(N, *b), grid_line_blocks(N, p), _xtrue(n, seed),
                    f"cd2d_{N}_p{p}", {"N": N, "b": tuple(b)})


def small_convdiff_3d(N: int, planes: list[int], b=(10.0, 20.0, 30.0), seed: int = 0) -> Problem:
    n = N ** 3
    return _problem(n, convdiff_3d(N, *b), slab_blocks(N, planes), _xtrue(n, seed),
                    f"cd3d_{N}_slabs{len(planes)}", {"N": N, "b": tuple(b), "planes": planes})


def small_random_band(n: int, p: int, hw: int, k_off: int = 11, p_long: float = 0.01,
                      dd: float = 1.2, seed: int = 0) -> Problem:
    rng = np.random.default_rng([seed, 4])
    csr = random_band(n, hw, k_off, p_long, dd, rng)
    return _problem(n, csr, equal_blocks(n, p), _xtrue(n, seed), f"randband_{n}_p{p}",
                    {"hw": hw, "k_off": k_off, "p_long": p_long, "dd": dd})


def small_random_dd(n: int, p: int, k_off: int = 4, dd: float = 1.5, seed: int = 0,
                    symmetric_pattern: bool = False) -> Problem:
    rng = np.random.default_rng([seed, 7])
    csr = random_dd(n, k_off, dd, rng, symmetric_pattern)
    return _problem(n, csr, equal_blocks(n, p), _xtrue(n, seed), f"randdd_{n}_p{p}",
                    {"k_off": k_off, "dd": dd})


def worked_example(A_dense: np.ndarray, block_ptr, f) -> Problem:
    """Wrap a small dense system (e.g. a printed example) as a CSR ``Problem``."""
    A_dense = np.asarray(A_dense, dtype=np.float64)
    n = A_dense.shape[0]
    r, c = np.nonzero(A_dense)
    rowptr, colind, values = _coo_to_csr(n, r.astype(np.int64), c.astype(np.int64), A_dense[r, c])
    return Problem(n=n, rowptr=rowptr, colind=colind, values=values,
                   block_ptr=np.asarray(block_ptr, dtype=np.int64), f=np.asarray(f, dtype=np.float64),
                   x_true=None, name="dense", meta={})
