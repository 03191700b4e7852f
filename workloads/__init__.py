"""Seeded synthetic linear systems shared by the CUDA solver's tests, the bench
and the CPU oracle.

This package only *builds inputs*: sparsity patterns, matrix values, block-row
partitions and right-hand sides. It holds none of the DDPS method's arithmetic
(no splitting, factorisation, spikes, reduced system or Krylov step), so the
oracle and the CUDA path can both take their inputs from it without sharing
any of the computation they are compared on.
"""

from .generate import (  # noqa: F401
    Problem,
    convdiff_2d,
    convdiff_3d,
    equal_blocks,
    grid_line_blocks,
    slab_blocks,
    random_band,
    random_dd,
    cfg1,
    cfg2,
    cfg2_slab_planes,
    cfg3,
    cfg3_sides,
    cfg4,
    cfg5,
    cfg5_coeff,
    small_convdiff_2d,
    small_convdiff_3d,
    small_random_band,
    small_random_dd,
    worked_example,
)
