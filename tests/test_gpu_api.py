"""GPU tests of the library's API beyond single-step parity: eigenvalue readout, state
save/restore, error reporting, and convergence of the whole iteration to the exact
solution (O1) on the 64-dimensional CCA workload."""
import numpy as np
import pytest

import synth
from oracle import gep

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2206_04993_gb300 import Solver, sgep as S  # noqa: E402

PATHS = [S.SGEP_PATH_GENERIC, S.SGEP_PATH_CLUSTER]
IDS = ["generic", "cluster"]


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(dtype)


@pytest.mark.parametrize("kind", ["cca", "pca", "pls"])
def test_eigenvalue_readout_matches_rayleigh_quotients(kind):
    """lambda_i = v_i^T A v_i / v_i^T B v_i on an evaluation batch (Sec. 2; App. H.2.2),
    with A, B formed by the oracle from the same rows; n spans several max_b chunks."""
    model = synth.planted_cca(30, 26, [0.9, 0.7, 0.5, 0.3], seed=4)
    X, Y = synth.draw_rows(model, 1000, batch=3)
    X32, Y32 = X.astype(np.float32), Y.astype(np.float32)
    V = synth.random_unit_columns(56 if kind != "pca" else 30, 3, seed=6).astype(np.float32)
    kw = dict(kind={"cca": S.SGEP_CCA, "pca": S.SGEP_PCA, "pls": S.SGEP_PLS}[kind], k=3,
              d_x=30, d_y=0 if kind == "pca" else 26, max_b=256)
    with Solver(**kw) as s:
        s.set_V(V)
        lam = s.eigenvalues(_dev(X32), None if kind == "pca" else _dev(Y32))
    if kind == "cca":
        A, B = gep.form_cca_AB(X32.astype(np.float64), Y32.astype(np.float64))
    elif kind == "pls":
        A, B = gep.form_pls_AB(X32.astype(np.float64), Y32.astype(np.float64))
    else:
        A, B = gep.form_pca_AB(X32.astype(np.float64))
    ref = gep.rayleigh_quotients(V.astype(np.float64), A, B)
    np.testing.assert_allclose(lam, ref, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("path", PATHS, ids=IDS)
def test_state_roundtrip_resumes_exactly(path):
    model = synth.planted_cca(40, 40, [0.9, 0.6, 0.3], seed=1)
    X, Y = synth.draw_rows(model, 128 * 20, batch=5)
    Xd, Yd = _dev(X), _dev(Y)
    kw = dict(kind=S.SGEP_CCA, d_x=40, d_y=40, k=3, eta0=0.2, gamma0=0.5, path=path,
              schedule=S.SGEP_SCHED_HOLD_HARMONIC, t_c=4, T=40, eta_T=0.02)
    with Solver(**kw) as a:
        a.step_many(Xd, Yd, 128, 20)
        Va = a.V()
    with Solver(**kw) as b, Solver(**kw) as c:
        b.step_many(Xd[:1280], Yd[:1280], 128, 10)
        blob = b.state()
        c.load_state(blob)
        assert c.t == 10
        c.step_many(Xd[1280:], Yd[1280:], 128, 10)
        Vc = c.V()
    assert np.linalg.norm(Vc - Va) / np.linalg.norm(Va) < 1e-5
    with Solver(kind=S.SGEP_CCA, d_x=40, d_y=41, k=3) as d:
        with pytest.raises(S.SgepError) as ei:
            d.load_state(blob)
        assert ei.value.status == S.SGEP_ESTATE
        with pytest.raises(S.SgepError):
            d.load_state(blob[:-4])


@pytest.mark.parametrize("path", PATHS, ids=IDS)
def test_nonfinite_input_is_reported(path):
    X = np.random.default_rng(0).standard_normal((64, 16)).astype(np.float32)
    Y = np.random.default_rng(1).standard_normal((64, 12)).astype(np.float32)
    X[5, 3] = np.nan
    with Solver(kind=S.SGEP_CCA, d_x=16, d_y=12, k=2, path=path) as s:
        s.step(_dev(X), _dev(Y))
        with pytest.raises(S.SgepError) as ei:
            s.V()
        assert ei.value.status == S.SGEP_ENONFINITE
        # the flag is cleared once reported; a clean state and batch work again
        s.set_V(synth.random_unit_columns(28, 2, seed=0).astype(np.float32))
        X[5, 3] = 0.0
        s.step(_dev(X), _dev(Y))
        assert np.isfinite(s.V()).all()


def test_step_argument_errors():
    with Solver(kind=S.SGEP_CCA, d_x=8, d_y=8, k=2, max_b=64) as s:
        X = _dev(np.zeros((65, 8)))
        with pytest.raises(S.SgepError) as ei:
            s.step(X, X)
        assert ei.value.status == S.SGEP_EINVAL
        with pytest.raises(S.SgepError):
            s.step(X[:1], X[:1])       # split batches need 2 rows
        with pytest.raises(S.SgepError):
            S.sgep_step(s.h, X, None, None, 8)   # CCA needs Y


def test_initial_V_has_unit_columns_and_S_equals_V():
    with Solver(kind=S.SGEP_PCA, d_x=300, d_y=0, k=7, seed=42) as s:
        V, Sm = s.V(), s.S()
    np.testing.assert_allclose(np.linalg.norm(V, axis=0), 1.0, atol=1e-6)
    np.testing.assert_array_equal(V, Sm)
    assert abs(V.mean()) < 0.05 and 0.5 < V.std() * np.sqrt(300) < 1.5


@pytest.mark.parametrize("path", PATHS, ids=IDS)
def test_small_cca_workload_converges_to_exact_solution(path):
    """Alg. 2 on the finite 10,000-row CCA set (d = 64, k = 4, b = 256, 2000 steps of
    with-replacement minibatches): generalized subspace error below 1e-3 and eigenvalue
    error below 1e-3 against Cholesky + Jacobi on the finite-sample A, B."""
    cfg = synth.config_c1()
    X, Y = cfg["X"], cfg["Y"]
    A, B = gep.form_cca_AB(X, Y)
    lam, Vs = gep.gep_topk(A, B, 4)
    steps = cfg["steps"]
    idx = np.concatenate([synth.finite_dataset_indices(10_000, 256, t) for t in range(1, steps + 1)])
    Xd, Yd = _dev(X), _dev(Y)
    it = torch.from_numpy(idx).cuda()
    Xb, Yb = Xd[it].contiguous(), Yd[it].contiguous()
    with Solver(kind=S.SGEP_CCA, d_x=32, d_y=32, k=4, eta0=cfg["eta0"], gamma0=cfg["gamma0"],
                rho=cfg["rho"], schedule=cfg["schedule"], t_c=cfg["t_c"], T=cfg["T"],
                eta_T=cfg["eta_T"], path=path, max_b=10_000) as s:
        s.set_V(synth.random_unit_columns(64, 4, seed=0).astype(np.float32))
        s.step_many(Xb, Yb, 256, steps)
        V = s.V().astype(np.float64)
        lam_hat = s.eigenvalues(Xd, Yd)
    err = gep.subspace_error(Vs, V, B)
    assert err < 1e-3, err
    assert np.max(np.abs(lam_hat - lam)) < 1e-3, (lam_hat, lam)
