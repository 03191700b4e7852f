"""DDPS (domain-decomposing parallel sparse solver, arXiv 1008.1700) on one
GB300 GPU: a C-ABI CUDA library (``include/ddps.h``) and this thin binding."""

from . import native  # noqa: F401
from .native import DDPSError  # noqa: F401
from .solver import Solver, stack_systems  # noqa: F401
