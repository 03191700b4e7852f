"""CPU checks of the native library: it loads, exports every entry point the
header declares, and its host-side symbolic analysis (Fig. 2 steps 1, 3, 5
and the nested-dissection layout) agrees with the oracle.  No GPU calls."""

import numpy as np
import pytest

import workloads as W
from oracle.ddps_oracle import DDPSOracle
from paper_1008_1700_gb300 import native as N
from paper_1008_1700_gb300.solver import stack_systems


def test_library_exports_every_declared_symbol():
    declared = N._declared_names()
    assert "ddps_analyze" in declared and "ddps_solve" in declared
    lib = N.load()
    missing = [d for d in declared if not hasattr(lib, d)]
    assert missing == []


CASES = [
    (lambda: W.cfg1(), None),
    (lambda: W.small_convdiff_3d(10, [3, 4, 3]), None),
    (lambda: W.small_random_band(3000, 5, 200, seed=2), ("abs", 1e-4)),
    (lambda: W.small_random_band(3000, 5, 200, seed=3), ("column", 0.6)),
    (lambda: W.small_random_dd(301, 7, seed=9), None),
]


def _opts(drop):
    if drop is None:
        return N.default_options()
    mode = N.DDPS_DROP_ABS if drop[0] == "abs" else N.DDPS_DROP_COLUMN
    return N.default_options(drop_mode=mode, drop_tol=drop[1])


@pytest.mark.parametrize("make,drop", CASES)
def test_symbolic_matches_oracle(make, drop):
    P = make()
    sizes, perm, c = N.ddps_symbolic(P.rowptr, P.colind, P.block_ptr, values=P.values,
                                     options=_opts(drop))
    o = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, drop=drop, spikes=False)
    # Fig. 2 step 5: the same interface set
    assert np.array_equal(c, o.c)
    assert sizes["m"] == o.m and sizes["nnz_rt"] == o.Rt.nnz
    # G^ layout: block rows in c times coupling columns
    assert sizes["ghat_entries"] == sum((b["q1"] - b["q0"]) * len(b["c_i"]) for b in o.blk)
    # the ordering permutes rows inside their own block only
    assert np.array_equal(np.sort(perm), np.arange(P.n))
    blk_of = np.searchsorted(P.block_ptr, np.arange(P.n), side="right") - 1
    assert np.array_equal(blk_of[perm], blk_of)


def test_symbolic_rejects_bad_input():
    P = W.small_random_dd(40, 2, seed=1)
    bad = P.colind.copy()
    bad[3] = P.n + 5
    with pytest.raises(N.DDPSError, match="INVALID_ARG"):
        N.ddps_symbolic(P.rowptr, bad, P.block_ptr)
    with pytest.raises(N.DDPSError, match="INVALID_ARG"):
        N.ddps_symbolic(P.rowptr, P.colind, np.array([0, 30, 20, 40]))
    with pytest.raises(N.DDPSError, match="INVALID_ARG"):  # drop rule without values
        N.ddps_symbolic(P.rowptr, P.colind, P.block_ptr,
                        options=N.default_options(drop_mode=N.DDPS_DROP_ABS, drop_tol=1e-3))


def test_stack_systems_and_cross_system_entries():
    a = W.small_convdiff_2d(6, 2)
    b = W.small_random_dd(30, 3, seed=4)
    rp, ci, v, bp, sbp, srp = stack_systems([(a.rowptr, a.colind, a.values, a.block_ptr),
                                             (b.rowptr, b.colind, b.values, b.block_ptr)])
    assert list(sbp) == [0, 2, 5] and list(srp) == [0, 36, 66]
    sizes, perm, c = N.ddps_symbolic(rp, ci, bp, sbp)
    ca = DDPSOracle(a.n, a.rowptr, a.colind, a.values, a.block_ptr, spikes=False).c
    cb = DDPSOracle(b.n, b.rowptr, b.colind, b.values, b.block_ptr, spikes=False).c
    assert np.array_equal(c, np.concatenate([ca, cb + a.n]))
    # an entry coupling the two systems is rejected
    ci2 = ci.copy()
    ci2[rp[1] - 1] = 40  # row 0 of system a pointing into system b
    ci2[rp[0]:rp[1]] = np.sort(ci2[rp[0]:rp[1]])
    with pytest.raises(N.DDPSError, match="couples two systems"):
        N.ddps_symbolic(rp, ci2, bp, sbp)


def test_analyze_rejects_bad_options_before_any_device_work():
    """Option checks run before the analysis touches the device, so they hold
    on a machine without a GPU."""
    P = W.small_random_dd(40, 2, seed=1)
    bad = [dict(update_prec=N.DDPS_BF16X3),  # tensor-core updates need FP32 factors
           dict(factor_prec=N.DDPS_FP32, update_prec=N.DDPS_BF16),
           dict(ghat_mode=2),
           dict(fused_rows=-2)]
    for kw in bad:
        with pytest.raises(N.DDPSError, match="INVALID_ARG"):
            N.ddps_analyze(P.rowptr, P.colind, P.block_ptr, options=N.default_options(**kw))


@pytest.mark.parametrize("make,drop", CASES[:3])
def test_symbolic_ilu_keeps_the_block_order(make, drop):
    """With ILU(0) block factors the blocks keep their own row order (the
    factor is defined on it); c and the G^ layout are those of the oracle."""
    P = make()
    o = _opts(drop)
    o.factor_kind = N.DDPS_FACTOR_ILU0
    o.factor_prec = o.spike_prec = N.DDPS_FP64
    sizes, perm, c = N.ddps_symbolic(P.rowptr, P.colind, P.block_ptr, values=P.values, options=o)
    assert np.array_equal(perm, np.arange(P.n))
    orc = DDPSOracle(P.n, P.rowptr, P.colind, P.values, P.block_ptr, drop=drop, spikes=False)
    assert np.array_equal(c, orc.c)
    assert sizes["nfronts"] == 0
    # a solve streams the stored entries of the diagonal blocks
    nnz_d = sum(Dii.nnz for Dii in orc.D_blocks)
    assert sizes["factor_lu_entries"] == nnz_d


@pytest.mark.parametrize("make,drop", [CASES[1], CASES[3]])
def test_symbolic_does_not_depend_on_the_thread_count(make, drop, monkeypatch):
    """The blocks are analysed in parallel; every block writes only its own
    part of the result, so one thread and several give the same analysis."""
    P = make()
    out = []
    for t in ("1", "3", "16"):
        monkeypatch.setenv("DDPS_ANALYZE_THREADS", t)
        out.append(N.ddps_symbolic(P.rowptr, P.colind, P.block_ptr, values=P.values,
                                   options=_opts(drop)))
    for sizes, perm, c in out[1:]:
        assert sizes == out[0][0]
        assert np.array_equal(perm, out[0][1]) and np.array_equal(c, out[0][2])


def test_threaded_analysis_reports_the_first_bad_entry(monkeypatch):
    """With entries coupling two systems in several blocks, the error names
    the first one in row order, whatever the thread count."""
    a = W.small_convdiff_2d(8, 4)
    b = W.small_random_dd(40, 4, seed=5)
    rp, ci, v, bp, sbp, srp = stack_systems([(a.rowptr, a.colind, a.values, a.block_ptr),
                                             (b.rowptr, b.colind, b.values, b.block_ptr)])
    ci2 = ci.copy()
    for row, col in ((a.n + 35, 3), (20, a.n + 7)):  # a row of b into a, a row of a into b
        e = rp[row + 1] - 1 if col > ci2[rp[row + 1] - 1] else rp[row]
        ci2[e] = col
        ci2[rp[row]:rp[row + 1]] = np.sort(ci2[rp[row]:rp[row + 1]])
    for t in ("1", "16"):
        monkeypatch.setenv("DDPS_ANALYZE_THREADS", t)
        with pytest.raises(N.DDPSError, match=rf"entry \(20, {a.n + 7}\) couples two systems"):
            N.ddps_symbolic(rp, ci2, bp, sbp)
