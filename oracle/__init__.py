"""Plain FP64 CPU oracle for the gamma-EigenGame hot path.

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the CPU
baseline leg of `bench.py` may import this package. The product (the CUDA
library and its Python binding) never imports, links or runs anything here,
and this package never imports the product.

Two parts:

* `oracle.gep`  (O1) -- the exact top-k solution of A v = lambda B v: Cholesky
  reduction, a cyclic Jacobi eigensolver, closed forms for the planted models,
  and the generalized subspace error (App. A, Prop. "Similar Matrices" and
  Sec. A.1).
* `oracle.eg`   (O2) -- the stochastic gamma-EigenGame iteration (Alg. 2, with
  M = 1) written player by player as the paper states it, the deterministic
  variant (Alg. 1), the utilities (Eq. util_new), the schedule of App. H, and
  the streamed minibatch mat-vec operators for CCA / PLS / PCA / LDA.

Every function works in float64. Parity status of each function is listed in
its module header; functions without an independent pin say "parity unpinned".
"""
from . import gep, eg  # noqa: F401
