"""GB300-native minibatch gamma-EigenGame for the top-k symmetric generalized
eigenproblem A v = lambda B v (arXiv 2206.04993, Alg. 2).

The computation lives in libsgep.so (CUDA, sm_103a) behind the C ABI of
include/sgep.h; `paper_2206_04993_gb300.sgep` binds it with ctypes and
`paper_2206_04993_gb300.solver.Solver` is a small convenience wrapper.
"""
from . import sgep  # noqa: F401
from .solver import Batch, Solver, WarmStart  # noqa: F401
