"""ddps_block_solve_noalloc: the block solve of Fig. 3 step 6.1 for callers
that cannot allocate device memory when they need it (a memory pool that
already owns all free device memory, or a policy of allocating only at
start-up).  Its scratch comes from a fixed 16 MiB array inside the library.
The test calls it through the C ABI twice in a row and compares each result
with ddps_block_solve on the same handle."""

import numpy as np
import pytest
import torch

import workloads as W
from gpu_helpers import dev, host, make_solver, relerr
from paper_1008_1700_gb300 import native as N

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [N.DDPS_FP64, N.DDPS_FP32])
def test_noalloc_block_solve_matches_block_solve(prec):
    P = W.small_convdiff_3d(12, [3, 5, 4])
    S = make_solver(P, factor_prec=prec, spike_prec=prec, ghat_prec=prec, inner_prec=prec)
    rng = np.random.default_rng(7)
    for call in range(2):  # the second call sees the first call's leftovers in the array
        y = dev(rng.standard_normal(P.n))
        g_ref = torch.empty_like(y)
        N.ddps_block_solve(S.h, y, g_ref)
        g = torch.full_like(y, float("nan"))
        N.ddps_block_solve_noalloc(S.h, y, g)
        assert relerr(host(g), host(g_ref)) <= 1e-12, call
    S.close()


def test_noalloc_rejects_problems_beyond_the_array():
    # one block of 1000^2 unknowns in FP64 needs about 19 MB of scratch
    # (8 MB for the permuted vector, 11 MB for the multifrontal update entries)
    P = W.small_convdiff_2d(1000, 1)
    S = make_solver(P)
    y = dev(np.ones(P.n))
    g = torch.empty_like(y)
    with pytest.raises(N.DDPSError, match="INVALID_ARG.*scratch"):
        N.ddps_block_solve_noalloc(S.h, y, g)
    S.close()
