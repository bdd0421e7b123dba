"""Alg. 2 with M > 1 machines on the GPU (generic path) against the oracle: every machine's
update direction and auxiliary increment from its own shard of the step's rows, averaged."""
import numpy as np
import pytest

import synth
from gpu_util import STEP_TOL, rel
from oracle import eg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2206_04993_gb300 import Solver, sgep as S  # noqa: E402


def _ops(kind, X, Y):
    if kind == "pca":
        return eg.pca_ops(X)
    if kind == "pls":
        return eg.pls_ops(X, Y)
    return eg.cca_ops(X, Y)


@pytest.mark.parametrize("kind,M,b", [("cca", 2, 512), ("cca", 3, 600), ("pca", 4, 256), ("pls", 2, 300)])
def test_machines_match_oracle_over_steps(kind, M, b):
    dx, dy, k, n = 40, (0 if kind == "pca" else 24), 5, 4
    model = synth.planted_cca(dx, max(dy, 1), np.linspace(0.9, 0.4, 8), seed=M + b)
    X, Y = synth.draw_rows(model, b * n, batch=3, dtype=np.float32)
    Y = None if kind == "pca" else Y[:, :dy]
    V0 = synth.random_unit_columns(dx + dy, k, seed=12).astype(np.float32)
    S0 = (0.8 * V0 + 0.05 * synth.random_unit_columns(dx + dy, k, seed=13)).astype(np.float32)
    kinds = {"cca": S.SGEP_CCA, "pca": S.SGEP_PCA, "pls": S.SGEP_PLS}
    with Solver(kind=kinds[kind], d_x=dx, d_y=dy, k=k, machines=M, eta0=0.3, gamma0=0.4, rho=1e-3,
                max_b=b) as s:
        assert s.path == S.SGEP_PATH_GENERIC
        s.set_V(V0, S0)
        Xd = torch.from_numpy(X).cuda()
        Yd = None if Y is None else torch.from_numpy(np.ascontiguousarray(Y)).cuda()
        s.step_many(Xd, Yd, b, n)
        s.sync()
        Vg, Sg = s.V(), s.S()
    V, Sv = V0.astype(np.float64), S0.astype(np.float64)
    X64 = X.astype(np.float64)
    Y64 = None if Y is None else Y.astype(np.float64)
    for t in range(n):
        rows = [slice(t * b + b * m // M, t * b + b * (m + 1) // M) for m in range(M)]
        ops = [_ops(kind, X64[r], None if Y64 is None else Y64[r]) for r in rows]
        V, Sv = eg.eg_step_machines(V, Sv, ops, 0.3, 0.4, 1e-3)
    ev, es = rel(Vg, V), rel(Sg, Sv)
    print({"V": ev, "S": es})
    assert ev < n * STEP_TOL and es < n * STEP_TOL


def test_machines_need_generic_path_and_plain_step():
    with pytest.raises(S.SgepError):
        Solver(kind=S.SGEP_CCA, d_x=512, d_y=512, k=8, dtype=S.SGEP_BF16, path=S.SGEP_PATH_TC, machines=2)
    with pytest.raises(S.SgepError):
        Solver(kind=S.SGEP_CCA, d_x=16, d_y=16, k=2, machines=2, optimizer=S.SGEP_OPT_ADAM)
    with pytest.raises(S.SgepError):
        Solver(kind=S.SGEP_CCA, d_x=16, d_y=16, k=2, machines=0)
    with Solver(kind=S.SGEP_CCA, d_x=16, d_y=16, k=2, machines=4, max_b=64) as s:
        X = torch.zeros(6, 16, device="cuda")  # 6 rows cannot give 4 machines a split batch each
        with pytest.raises(S.SgepError):
            s.step(X, X)
