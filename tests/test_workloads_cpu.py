"""The synthetic workloads match the recipes they stand for: sizes,
partitions, value structure (convection-diffusion stencils scaled by h^2,
the random band's diagonal dominance and band), and f = A x_true.  CPU."""

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W


def _csr(P):
    return sp.csr_matrix((P.values, P.colind, P.rowptr), shape=(P.n, P.n))


def test_cd2d_64_p4():
    P = W.cfg1()
    assert (P.n, P.nnz, P.p) == (4096, 20224, 4)
    assert list(np.diff(P.block_ptr)) == [1024] * 4
    A = _csr(P)
    # 5-point stencil scaled by h^2: diagonal 4, neighbours -1 -+ b h / 2
    h = 1.0 / 65
    assert np.allclose(A.diagonal(), 4.0)
    off = A - sp.diags(A.diagonal())
    vals = np.unique(np.round(off.data, 12))
    assert np.allclose(sorted(vals), sorted({round(-1 - 10 * h / 2, 12), round(-1 + 10 * h / 2, 12)}))
    assert np.allclose(A @ P.x_true, P.f)
    assert np.all(np.abs(P.x_true) <= 1.0)


def test_cd3d_64_slabs16():
    P = W.cfg2()
    assert (P.n, P.nnz, P.p) == (262144, 1810432, 16)
    planes = np.diff(P.block_ptr) // (64 * 64)
    assert np.all(np.diff(P.block_ptr) % (64 * 64) == 0)
    assert planes.sum() == 64 and planes.min() >= 3 and planes.max() <= 5
    A = _csr(P)
    assert np.allclose(A.diagonal(), 6.0)
    # an M-matrix: non-positive off-diagonals (b h / 2 < 1)
    off = A - sp.diags(A.diagonal())
    assert off.data.max() <= 0.0
    assert np.allclose(A @ P.x_true, P.f)


def test_cd2d_batch256():
    probs = W.cfg3()
    assert len(probs) == 256
    assert sum(p.n for p in probs) == 1860814 and sum(p.nnz for p in probs) == 9221614
    sides = np.sqrt([p.n for p in probs]).astype(int)
    assert sides.min() >= 32 and sides.max() <= 128
    assert all(p.p == 8 for p in probs)


def test_cd3d_48_sequence():
    P = W.cfg5(1)
    assert (P.n, P.nnz, P.p) == (110592, 760320, 8)
    assert list(np.diff(P.block_ptr)) == [6 * 48 * 48] * 8
    assert W.cfg5_coeff(50) == pytest.approx(30.0)
    assert W.cfg5_coeff(150) == pytest.approx(10.0)


def test_random_band_1m():
    P = W.cfg4()
    assert (P.n, P.nnz, P.p) == (1_000_000, 12_000_000, 128)
    assert np.array_equal(P.block_ptr, [(i * P.n) // 128 for i in range(129)])
    A = _csr(P)
    d = A.diagonal()
    offsum = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(d)
    assert np.allclose(np.abs(d), 1.2 * offsum)
    coo = A.tocoo()
    far = np.abs(coo.row - coo.col) > 2000
    # about 1% of the off-diagonal entries reach beyond the band
    frac = far.sum() / (A.nnz - P.n)
    assert 0.002 < frac < 0.03
    assert np.allclose(A @ P.x_true, P.f)
