"""B300-native batched Safety-Filter (SF) solver of Flow-Opt (arXiv 2510.09204).

The solver runs in ``libsf.so`` (hand-written CUDA for sm_103a behind the C ABI in
``include/sf.h``); this package is its Python binding.
"""
from .sf import (SFSolver, SFSolve, SFError, lib, PRECISIONS, PROJECTIONS, EXPORTS,  # noqa: F401
                 SF_RES_RP, SF_RES_MAX, SF_RES_FP, SF_RES_ITERS, SF_RES_FPSUM, SF_NRES)

__version__ = "0.1.0"
