"""Parity at the full workload sizes, in the configuration bench.py times
(its ``form_options("mixed")``: FP32 factors, bf16x3 tensor-core spike
products and LU block updates, FP16 G^, FP64 outer): the oracle's solution
x = A^-1 f (stored by tests/golden/make_fullsize_reference.py as norms and
sampled entries), properties that hold at any size (recomputed residual,
error against the known solution) for every system, and sampled outputs the
oracle computes one at a time (spike columns G_i(:, k) = A_ii^-1 R~_i(:, k)
restricted to the rows in c, and whole systems of the batch)."""

import json
import os

import numpy as np
import pytest
import torch

import bench
import workloads as W
from gpu_helpers import dev, host, relerr
from oracle.ddps_oracle import DDPSOracle, csr
from paper_1008_1700_gb300 import Solver, native as N

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

# exactly the options bench.py times (tolerances included)
BENCH_FORM = bench.form_options("mixed")

_REF = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    "fullsize_reference.json")


def _check_against_oracle_x(name, x, bound=1e-8):
    """x against the oracle's stored solution: relative error of the sampled
    entries and of the 2-norm."""
    with open(_REF) as fh:
        ref = json.load(fh)[name]
    assert len(x) == ref["n"]
    idx = np.asarray(ref["idx"])
    xr = np.asarray(ref["x"])
    assert relerr(x[idx], xr) <= bound, name
    assert abs(np.linalg.norm(x) - ref["norm2"]) <= bound * ref["norm2"], name


def _check_sampled_spikes(S, P, o, blocks, ncols, rng, tol):
    """GPU G^ rows of block b against oracle spike columns."""
    for b in blocks:
        q0, q1, cols = S.ghat_layout(b)
        if len(cols) == 0 or q1 == q0:
            continue
        Gg = S.ghat_block(b)
        ob = o.blk[b]
        for j in rng.choice(len(cols), size=min(ncols, len(cols)), replace=False):
            k = int(o.c[cols[j]])
            col = o.spike_column(b, k)[ob["rows_c"]]
            scale = max(np.max(np.abs(col)), 1e-300)
            assert np.max(np.abs(Gg[:, j] - col)) <= tol * scale, (b, j)


def _solve(P, **opts):
    S = Solver(P.rowptr, P.colind, P.block_ptr, **opts)
    S.factor(dev(P.values))
    x, info = S.solve(dev(P.f))
    return S, host(x), info


def test_cd3d_64_slabs16_bench_configuration():
    P = W.cfg2()
    S, x, info = _solve(P, **BENCH_FORM)
    A = csr(P.n, P.rowptr, P.colind, P.values)
    rr = np.max(np.abs(P.f - A @ x)) / np.max(np.abs(P.f))
    assert info["status"] == "DDPS_OK" and rr <= 1e-10
    assert relerr(x, P.x_true) <= 1e-8
    _check_against_oracle_x("cd3d_64_slabs16", x)
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, spikes=False)
    _check_sampled_spikes(S, P, o, blocks=(0, 7, 15), ncols=4, rng=np.random.default_rng(0),
                          tol=2e-3)  # FP16 storage of G^
    S.close()


def test_cd3d_64_slabs16_plain_fp64():
    P = W.cfg2()
    S, x, info = _solve(P, factor_prec=N.DDPS_FP64, spike_prec=N.DDPS_FP64,
                        ghat_prec=N.DDPS_FP64, inner_prec=N.DDPS_FP64, tol_out=1e-12,
                        tol_in=1e-4)
    A = csr(P.n, P.rowptr, P.colind, P.values)
    assert info["status"] == "DDPS_OK"
    assert np.max(np.abs(P.f - A @ x)) / np.max(np.abs(P.f)) <= 1e-12
    assert relerr(x, P.x_true) <= 1e-9
    _check_against_oracle_x("cd3d_64_slabs16", x, bound=1e-9)
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, spikes=False)
    _check_sampled_spikes(S, P, o, blocks=(3, 12), ncols=3, rng=np.random.default_rng(1), tol=1e-10)
    S.close()


def test_batch_256_systems_full_size():
    probs = W.cfg3()
    S = Solver.from_systems([(p.rowptr, p.colind, p.values, p.block_ptr) for p in probs],
                            **BENCH_FORM)
    S.factor(dev(S.values_host))
    x, info = S.solve(dev(np.concatenate([p.f for p in probs])))
    x = host(x)
    assert info["status"] == "DDPS_OK"
    for k, p in enumerate(probs):
        xk = x[S.sys_row_ptr[k]:S.sys_row_ptr[k + 1]]
        A = csr(p.n, p.rowptr, p.colind, p.values)
        assert np.max(np.abs(p.f - A @ xk)) / np.max(np.abs(p.f)) <= 1e-10, k
        assert relerr(xk, p.x_true) <= 1e-7, k
    for k in (0, 99, 255):
        p = probs[k]
        xo, _ = DDPSOracle(p.n, p.rowptr, p.colind, p.values, p.block_ptr).solve(
            p.f, tol=1e-12, eps_in=1e-8)
        assert relerr(x[S.sys_row_ptr[k]:S.sys_row_ptr[k + 1]], xo) <= 1e-8, k
    S.close()


@pytest.mark.parametrize("t", [1, 150])
def test_cd3d_48_time_steps(t):
    P = W.cfg5(t)
    S, x, info = _solve(P, **BENCH_FORM)
    A = csr(P.n, P.rowptr, P.colind, P.values)
    assert info["status"] == "DDPS_OK"
    assert np.max(np.abs(P.f - A @ x)) / np.max(np.abs(P.f)) <= 1e-10
    _check_against_oracle_x(f"cd3d_48_t{t}", x)
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, spikes=False)
    _check_sampled_spikes(S, P, o, blocks=(0, 4, 7), ncols=3, rng=np.random.default_rng(t), tol=2e-3)
    z, g = S.reduced_solution()
    # the first application's reduced right-hand side is (D^-1 f)(c); FP32 block
    # factors bound its error by about cond(A_ii) * 2^-24 (cond(A_ii) ~ 1e2 here)
    assert relerr(host(g), o.block_solve(P.f)[o.c]) <= 1e-5
    S.close()


def test_random_band_1m_dropping():
    """1M-row random band, 128 blocks, element-wise drop |r_ij| < 1e-4: residual
    and error on the whole system; spike columns of three blocks against the
    oracle's LU of those blocks alone."""
    from oracle.ddps_oracle import drop_entries, factor_blocks, interface_columns, split_block_rows
    P = W.cfg4()
    S = Solver(P.rowptr, P.colind, P.block_ptr, values_host=P.values,
               **dict(BENCH_FORM, drop_mode=N.DDPS_DROP_ABS, drop_tol=1e-4))
    S.factor(dev(P.values))
    x, info = S.solve(dev(P.f))
    x = host(x)
    A = csr(P.n, P.rowptr, P.colind, P.values)
    assert info["status"] == "DDPS_OK"
    assert np.max(np.abs(P.f - A @ x)) / np.max(np.abs(P.f)) <= 1e-10
    assert relerr(x, P.x_true) <= 1e-8
    _check_against_oracle_x("randband_1m", x)
    D, R = split_block_rows(A, P.block_ptr)
    Rt = drop_entries(R, 1e-4)
    c = interface_columns(Rt)
    assert np.array_equal(S.interface(), c)
    rng = np.random.default_rng(4)
    for b in (0, 64, 127):
        r0, r1 = int(P.block_ptr[b]), int(P.block_ptr[b + 1])
        lu = factor_blocks([D[b]])[0]
        q0, q1, cols = S.ghat_layout(b)
        Gg = S.ghat_block(b)
        rows_c = c[(c >= r0) & (c < r1)] - r0
        Rb = Rt[r0:r1, :].tocsc()
        for j in rng.choice(len(cols), size=3, replace=False):
            colv = lu.solve(Rb[:, [int(c[cols[j]])]].toarray().ravel())[rows_c]
            scale = max(np.max(np.abs(colv)), 1e-300)
            assert np.max(np.abs(Gg[:, j] - colv)) <= 2e-3 * scale, (b, j)
    S.close()
