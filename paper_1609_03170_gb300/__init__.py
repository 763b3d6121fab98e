"""GB300-native open GRAPE without matrix exponentials (arXiv:1609.03170).

The hot path - RK4 propagation of the density matrix under the Lindblad
equation, the adjoint propagation under the dual Lindbladian and the
per-slice gradient traces - runs as hand-written sm_103a CUDA kernels behind
the C ABI of ``include/grape.h`` (``libgrape.so``).  This package holds the
build script, the ctypes binding and the problem front end.
"""
from . import _lib
from ._lib import (GRAPE_GRAD_EXACT, GRAPE_GRAD_FIRST_ORDER, GRAPE_PREC_DF64, GRAPE_PREC_FP64,
                   GrapeError, grape_forward,
                   grape_gradient, grape_problem_create, grape_problem_destroy)
from .problem import (BandModel, BandOp, GaussianFilter, GrapeBatch, GrapeProblem, GrapeServer,
                      band_model)


def __getattr__(name):
    # torch is imported only when the autograd front end is used
    if name in ("GrapeFunction", "grape_phi", "FilterFunction", "gaussian_filter"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)

__all__ = ["GRAPE_GRAD_EXACT", "GRAPE_GRAD_FIRST_ORDER", "GRAPE_PREC_DF64", "GRAPE_PREC_FP64",
           "GrapeError", "GrapeProblem", "GrapeBatch", "GrapeServer", "GaussianFilter",
           "BandModel", "BandOp", "band_model", "grape_forward", "grape_gradient",
           "grape_problem_create", "grape_problem_destroy"]
