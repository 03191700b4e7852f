"""Learned initial guess for the reduced solve (6.3) on a short time sequence
of 3-D convection-diffusion systems whose convection coefficient varies
smoothly: networks trained (by the library's kernels) on the reduced
solutions of the first half must cut the first application's inner
iterations on the second half, whose coefficients lie outside the training
range, against the paper's zero start and against the previous step's
reduced solution as the start (the honest baseline of a time sequence); every
solve still meets the outer tolerance."""

import numpy as np
import pytest

import workloads as W
from paper_1008_1700_gb300 import native as N
from paper_1008_1700_gb300.learned import run_sequence

pytestmark = pytest.mark.gpu


def test_learned_guess_cuts_inner_iterations():
    period = 40
    coeff = lambda t: 20.0 + 10.0 * np.sin(2 * np.pi * t / period)  # noqa: E731

    def make(t):
        P = W.small_convdiff_3d(20, [5, 5, 5, 5], b=(coeff(t),) * 3)
        P.f = np.full(P.n, 1.0 / 21 ** 2)
        return P

    opts = dict(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_BF16X3, ghat_prec=N.DDPS_FP32,
                inner_prec=N.DDPS_FP32, tol_out=1e-10, tol_in=1e-4, maxit_in=100)
    st = run_sequence(make, coeff, list(range(1, 21)), list(range(21, 41)), opts,
                      modes=("zero", "warm", "mlp", "mlp_warm"), fit_iters=1500, lr=1e-3)
    ev = st["eval"]
    for mode in ev:
        assert ev[mode]["relres_max"] <= 1e-10, mode
    assert ev["mlp"]["first_inner"] < ev["zero"]["first_inner"]
    assert ev["mlp_warm"]["first_inner"] < 0.85 * ev["zero"]["first_inner"]
    # the step-change network beats starting from the previous step's z^
    assert ev["mlp_warm"]["first_inner"] < ev["warm"]["first_inner"], ev
