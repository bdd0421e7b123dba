"""GPU parity: the library's CUDA path against the FP64 oracle on identical seeded inputs.

One step from an identical, unconverged state (so the update is not dominated by
cancellation) is compared term by term: A_t V and B_t V (the minibatch products), the
k x k terms, the update direction and the new V and [Bv]. The bar for FP32 is a relative
error of 1e-5 (update direction relative to the magnitude of its reward and penalty
terms). Shapes cover several tiles with ragged tails, single players, odd batch sizes and
the full 1024-dimensional workload."""
import numpy as np
import pytest

import synth
from gpu_util import STEP_TOL, assert_within, step_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2206_04993_gb300 import Solver, sgep as S  # noqa: E402

KINDS = {"pca": S.SGEP_PCA, "cca": S.SGEP_CCA, "pls": S.SGEP_PLS}


def _data(kind, dx, dy, b, seed):
    rng = np.random.default_rng(seed)
    if kind == "pca":
        model = synth.planted_pca(dx, np.linspace(4, 1, min(8, dx)), seed=seed)
        return synth.draw_pca_rows(model, b, batch=seed), None
    r = max(1, min(8, dx, dy))
    model = synth.planted_cca(dx, dy, np.linspace(0.9, 0.3, r), seed=seed)
    X, Y = synth.draw_rows(model, b, batch=seed)
    return X + 0.1 * rng.standard_normal(X.shape), Y


def _state(d, k, seed, kind):
    V = synth.random_unit_columns(d, k, seed=seed)
    # [Bv] away from B v so that every clipped and penalty term is exercised
    S_ = V * 0.8 + 0.05 * synth.random_unit_columns(d, k, seed=seed + 1)
    return V, S_


def _solver(kind, dx, dy, k, path, dtype="f32", **kw):
    try:
        return Solver(kind=KINDS[kind], d_x=dx, d_y=(0 if kind == "pca" else dy), k=k,
                      dtype=S.SGEP_BF16 if dtype == "bf16" else S.SGEP_F32, path=path,
                      debug=1, max_b=kw.pop("max_b", 4096), **kw)
    except S.SgepError as e:
        if e.status == S.SGEP_ENOTSUP and path != S.SGEP_PATH_GENERIC:
            pytest.skip(f"path {path} does not take this shape: {e}")
        raise


PATHS = [S.SGEP_PATH_GENERIC, S.SGEP_PATH_CLUSTER]


SHAPES = [
    # kind, d_x, d_y, k, b
    ("cca", 32, 32, 4, 256),
    ("cca", 512, 512, 16, 1024),
    ("cca", 37, 29, 3, 101),
    ("cca", 5, 3, 1, 2),
    ("cca", 70, 130, 17, 333),
    ("cca", 300, 200, 64, 64),
    ("cca", 1000, 24, 8, 67),
    ("pca", 100, 0, 5, 77),
    ("pca", 1, 0, 1, 9),
    ("pls", 40, 60, 6, 50),
]


@pytest.mark.parametrize("path", PATHS, ids=["generic", "cluster"])
@pytest.mark.parametrize("kind,dx,dy,k,b", SHAPES)
def test_single_step_matches_oracle(kind, dx, dy, k, b, path):
    X, Y = _data(kind, dx, dy, b, seed=dx + 7 * k + b)
    d = dx + (0 if kind == "pca" else dy)
    V0, S0 = _state(d, k, seed=b, kind=kind)
    with _solver(kind, dx, dy, k, path, eta0=0.3, gamma0=0.4, rho=1e-3) as s:
        err = step_errors(s, V0, S0, X, Y, kind, 0.3, 0.4, 1e-3)
    assert_within(err, STEP_TOL)


@pytest.mark.parametrize("kind,dx,dy,k,b", [("cca", 2048, 2048, 8, 8192), ("cca", 2046, 2050, 7, 8192),
                                             ("pls", 2048, 1024, 12, 8192)])
def test_generic_ring_many_stages_matches_oracle(kind, dx, dy, k, b):
    """Many row tiles make the projection take 1024-column chunks (32 stages of the cp.async
    ring, which wraps its slots eight times) and the back-projection ~50-stage row splits;
    row pitches that are and are not a multiple of 4 take the 16-byte and 4-byte copies."""
    X, Y = _data(kind, dx, dy, b, seed=dx + k)
    V0, S0 = _state(dx + dy, k, seed=k, kind=kind)
    with _solver(kind, dx, dy, k, S.SGEP_PATH_GENERIC, eta0=0.3, gamma0=0.4, rho=1e-3, max_b=b) as s:
        err = step_errors(s, V0, S0, X, Y, kind, 0.3, 0.4, 1e-3)
    assert_within(err, STEP_TOL)


@pytest.mark.parametrize("path", PATHS, ids=["generic", "cluster"])
def test_single_step_shared_batch_and_ridge(path):
    X, Y = _data("cca", 48, 40, 200, seed=3)
    V0, S0 = _state(88, 6, seed=5, kind="cca")
    with _solver("cca", 48, 40, 6, path, eta0=0.2, gamma0=1.0, rho=1e-6, split_AB=0, eps_B=0.05) as s:
        err = step_errors(s, V0, S0, X, Y, "cca", 0.2, 1.0, 1e-6, split=False, eps_B=0.05)
    assert_within(err, STEP_TOL)


@pytest.mark.parametrize("path", PATHS, ids=["generic", "cluster"])
@pytest.mark.parametrize("dx,dy,k,b", [(512, 512, 16, 1024), (160, 96, 6, 200), (64, 64, 4, 256)])
def test_single_step_bf16_aligned_shapes(path, dx, dy, k, b):
    """BF16 rows whose slices start on 16-byte boundaries (the asynchronous-copy path)."""
    X, Y = _data("cca", dx, dy, b, seed=dx + k)
    V0, S0 = _state(dx + dy, k, seed=4, kind="cca")
    with _solver("cca", dx, dy, k, path, dtype="bf16", eta0=0.3, gamma0=0.5, rho=1e-4) as s:
        err = step_errors(s, V0, S0, X, Y, "cca", 0.3, 0.5, 1e-4, dtype="bf16")
    assert_within(err, STEP_TOL)


@pytest.mark.parametrize("dx,dy,k,b", [(37, 29, 3, 101), (70, 130, 17, 333), (515, 301, 16, 640)])
def test_single_step_bf16_unaligned_rows(dx, dy, k, b):
    """BF16 rows whose length is odd or not a multiple of 8, on the generic path: each thread
    stages the aligned value pairs holding its values; the last pair of the matrix is read
    directly."""
    X, Y = _data("cca", dx, dy, b, seed=dx + dy)
    V0, S0 = _state(dx + dy, k, seed=6, kind="cca")
    with _solver("cca", dx, dy, k, S.SGEP_PATH_GENERIC, dtype="bf16", eta0=0.3, gamma0=0.5, rho=1e-4) as s:
        err = step_errors(s, V0, S0, X, Y, "cca", 0.3, 0.5, 1e-4, dtype="bf16")
    assert_within(err, STEP_TOL)


@pytest.mark.parametrize("path", PATHS, ids=["generic", "cluster"])
def test_single_step_bf16_inputs(path):
    """BF16 minibatch values (the GPU reads bf16, the oracle the same values in FP64);
    accumulation is FP32, so the same bar applies."""
    X, Y = _data("cca", 96, 80, 160, seed=9)
    V0, S0 = _state(176, 8, seed=2, kind="cca")
    with _solver("cca", 96, 80, 8, path, dtype="bf16", eta0=0.3, gamma0=0.5, rho=1e-4) as s:
        err = step_errors(s, V0, S0, X, Y, "cca", 0.3, 0.5, 1e-4, dtype="bf16")
    assert_within(err, STEP_TOL)


@pytest.mark.parametrize("path", PATHS, ids=["generic", "cluster"])
def test_clipping_active(path):
    """<v_j, [Bv]_j> below rho for some players: the clipped denominator is used."""
    X, Y = _data("cca", 20, 20, 64, seed=4)
    V0, _ = _state(40, 5, seed=8, kind="cca")
    S0 = -0.5 * V0
    with _solver("cca", 20, 20, 5, path, eta0=0.05, gamma0=0.3, rho=0.2) as s:
        err = step_errors(s, V0, S0, X, Y, "cca", 0.05, 0.3, 0.2)
    assert_within(err, STEP_TOL)


@pytest.mark.parametrize("path", PATHS, ids=["generic", "cluster"])
def test_twenty_steps_track_oracle(path):
    """Twenty consecutive steps on the 64-dimensional workload stay within 1e-4 of the
    oracle run on the same minibatch sequence (FP32 rounding compounds slowly)."""
    from oracle import eg
    cfg = synth.config_c1()
    Xall, Yall = cfg["X"].astype(np.float32), cfg["Y"].astype(np.float32)
    V = synth.random_unit_columns(64, 4, seed=0)
    Vr, Sr = V.astype(np.float64), V.astype(np.float64)
    with _solver("cca", 32, 32, 4, path, eta0=cfg["eta0"], gamma0=cfg["gamma0"], rho=cfg["rho"]) as s:
        s.set_V(V.astype(np.float32))
        for t in range(1, 21):
            idx = synth.finite_dataset_indices(10_000, 256, t)
            X, Y = Xall[idx], Yall[idx]
            s.step(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
            Vr, Sr = eg.eg_step(Vr, Sr, *eg.cca_ops(X, Y), cfg["eta0"], cfg["gamma0"], cfg["rho"])
        Vg, Sg = s.V(), s.S()
        assert s.t == 20
    assert np.linalg.norm(Vg - Vr) / np.linalg.norm(Vr) < 1e-4
    assert np.linalg.norm(Sg - Sr) / np.linalg.norm(Sr) < 1e-4


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_cluster_and_generic_paths_agree_over_many_steps(dtype):
    """The fused cluster kernel defers each update into the next launch; 200 steps of both
    paths on the same minibatches stay within 1e-4 of each other."""
    model = synth.planted_cca(160, 96, np.linspace(0.9, 0.4, 8), seed=2)
    X, Y = synth.draw_rows(model, 64 * 200, batch=77)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    Yd = torch.from_numpy(Y.astype(np.float32)).cuda()
    if dtype == "bf16":
        Xd, Yd = Xd.to(torch.bfloat16), Yd.to(torch.bfloat16)
    V0 = synth.random_unit_columns(256, 6, seed=1).astype(np.float32)
    out = {}
    for path in PATHS:
        with _solver("cca", 160, 96, 6, path, dtype=dtype, eta0=0.2, gamma0=0.5, rho=1e-6) as s:
            s.set_V(V0)
            s.step_many(Xd, Yd, 64, 200)
            out[path] = (s.V(), s.S(), s.t)
    (Vg, Sg, tg), (Vc, Sc, tc) = out[PATHS[0]], out[PATHS[1]]
    assert tg == tc == 200
    assert np.linalg.norm(Vc - Vg) / np.linalg.norm(Vg) < 1e-4
    assert np.linalg.norm(Sc - Sg) / np.linalg.norm(Sg) < 1e-4


@pytest.mark.parametrize("path", PATHS, ids=["generic", "cluster"])
def test_two_steps_then_read_matches_oracle(path):
    """Pending updates are completed by the next step and by the read."""
    from oracle import eg
    X, Y = _data("cca", 40, 30, 96, seed=12)
    V0, S0 = _state(70, 5, seed=3, kind="cca")
    with _solver("cca", 40, 30, 5, path, eta0=0.15, gamma0=0.6, rho=1e-5) as s:
        s.set_V(V0.astype(np.float32), S0.astype(np.float32))
        Xd = torch.from_numpy(X.astype(np.float32)).cuda()
        Yd = torch.from_numpy(Y.astype(np.float32)).cuda()
        s.step(Xd[:48], Yd[:48])
        s.step(Xd[48:], Yd[48:])
        Vg, Sg = s.V(), s.S()
    X32, Y32 = X.astype(np.float32), Y.astype(np.float32)
    V1, S1 = eg.eg_step(V0.astype(np.float32).astype(np.float64), S0.astype(np.float32).astype(np.float64),
                        *eg.cca_ops(X32[:48], Y32[:48]), 0.15, 0.6, 1e-5)
    V2, S2 = eg.eg_step(V1, S1, *eg.cca_ops(X32[48:], Y32[48:]), 0.15, 0.6, 1e-5)
    assert np.linalg.norm(Vg - V2) / np.linalg.norm(V2) < STEP_TOL * 3
    assert np.linalg.norm(Sg - S2) / np.linalg.norm(S2) < STEP_TOL * 3
