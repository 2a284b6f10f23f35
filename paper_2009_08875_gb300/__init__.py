"""GB300 space-time Schur-complement PCG for the heat equation (arXiv 2009.08875).

The solver lives in the CUDA library libst.so (C ABI in include/st.h).  `Solver` is a thin
ctypes wrapper whose methods take torch CUDA float64 tensors; it never computes anything
itself and raises if the library has not been built.
"""
from .solver import Batch, Server, Solver, STError, probe_fma_rates  # noqa: F401
