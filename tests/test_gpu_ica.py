"""GPU parity of the ICA kind (Sec. 1) against the FP64 oracle: one step from an identical
state (split quarters and unsplit, FP32 and BF16 rows), a short chained trajectory, and
convergence on streamed mixtures towards the population unmixing directions."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import synth  # noqa: E402
from gpu_util import bf16_round, rel, to_device  # noqa: E402
from oracle import eg, gep  # noqa: E402
from paper_2206_04993_gb300 import Solver  # noqa: E402
from paper_2206_04993_gb300 import sgep as S  # noqa: E402

LAWS = ["sparse"] * 4 + ["uniform"] * 6 + ["rademacher"] * 4 + ["gauss"] * 2
# ICA's A_t = K - tr(B) B - 2 B^2 cancels terms of size ~ d B down to ~ kappa B, so FP32 sums
# carry errors relative to the kurtosis term K (not to A_t): A_t V is checked against that scale.
TOL = 1e-5


def _step(split, dtype, b=1024, k=4, seed=4):
    model = synth.planted_ica(16, LAWS, seed=seed)
    X = synth.draw_ica_rows(model, b, batch=9)
    Xv = bf16_round(X) if dtype == "bf16" else np.asarray(X, np.float32)
    V0 = synth.random_unit_columns(16, k, seed=2)
    S0 = 0.8 * V0 + 0.05 * synth.random_unit_columns(16, k, seed=3)
    with Solver(kind=S.SGEP_ICA, d_x=16, d_y=0, k=k, dtype=S.SGEP_BF16 if dtype == "bf16" else S.SGEP_F32,
                eta0=0.01, gamma0=0.3, rho=1e-6, split_AB=1 if split else 0, max_b=b, debug=1) as s:
        assert s.path == S.SGEP_PATH_GENERIC
        s.set_V(V0.astype(np.float32), S0.astype(np.float32))
        s.step(to_device(Xv, dtype))
        AVg, BVg = s.products()
        Vg, Sg = s.V(), s.S()
    Amv, Bmv = eg.ica_ops(Xv, split=split)
    V1, S1, parts = eg.eg_step(V0.astype(np.float32).astype(np.float64), S0.astype(np.float32).astype(np.float64),
                               Amv, Bmv, 0.01, 0.3, 1e-6, return_parts=True)
    q = b // 4 if split else b
    X1 = np.asarray(Xv[:q], np.float64)
    w = np.einsum("rd,rd->r", X1, X1)
    kscale = np.linalg.norm((X1 * w[:, None]).T @ (X1 @ V0) / q)
    return {"AV": float(np.linalg.norm(AVg - parts["AV"]) / kscale), "BV": rel(BVg, parts["BV"]),
            "V": rel(Vg, V1), "S": rel(Sg, S1)}


@pytest.mark.parametrize("split,dtype", [(True, "f32"), (False, "f32"), (True, "bf16")])
def test_ica_single_step_matches_oracle(split, dtype):
    err = _step(split, dtype)
    print(err)
    for name, e in err.items():
        assert e <= TOL, (name, e, err)


def test_ica_trajectory_tracks_oracle():
    """Fifty chained steps on the same minibatches stay close to the FP64 iteration. One step
    agrees to ~1e-6; the early, noisy iteration amplifies that difference (measured: about
    1.15x per step, 8.6e-4 after 50 steps), so the bar for the trajectory is 5e-3."""
    model = synth.planted_ica(16, LAWS, seed=4)
    V = synth.random_unit_columns(16, 4, seed=1).astype(np.float32)
    Vr, Sr = V.astype(np.float64), V.astype(np.float64)
    with Solver(kind=S.SGEP_ICA, d_x=16, d_y=0, k=4, eta0=0.002, gamma0=0.3, rho=1e-6, max_b=1024) as s:
        s.set_V(V)
        for t in range(50):
            X = np.asarray(synth.draw_ica_rows(model, 1024, batch=300 + t), np.float32)
            s.step(to_device(X, "f32"))
            Vr, Sr = eg.eg_step(Vr, Sr, *eg.ica_ops(X), 0.002, 0.3, 1e-6)
        assert rel(s.V(), Vr) < 5e-3


def test_ica_converges_to_unmixing_directions():
    """Streamed mixtures: the players approach the top generalized eigenvectors of the
    population pencil (rows of M^-1 of the positive-kurtosis sources), and the Rayleigh
    quotients on a large evaluation batch approach kappa_j |m_j|^2."""
    model = synth.planted_ica(16, LAWS, seed=4)
    A, B = gep.ica_population_AB(model)
    lam, Vt = gep.gep_topk(A, B, 4)
    b = 1024
    with Solver(kind=S.SGEP_ICA, d_x=16, d_y=0, k=4, eta0=0.002, gamma0=0.3, rho=1e-6, max_b=8192,
                schedule=S.SGEP_SCHED_HOLD_HARMONIC, t_c=1, T=4001, eta_T=0.002 * 200.0 / 4200.0) as s:
        err0 = gep.subspace_error(Vt, s.V().astype(np.float64), B)
        for t0 in range(0, 4000, 200):
            X = np.asarray(synth.draw_ica_rows(model, 200 * b, batch=1000 + t0), np.float32)
            s.step_many(to_device(X, "f32"), None, b, 200)
        err = gep.subspace_error(Vt, s.V().astype(np.float64), B)
        Xe = np.asarray(synth.draw_ica_rows(model, 8192, batch=99), np.float32)
        lam_hat = s.eigenvalues(to_device(Xe, "f32"))
    print("subspace error", err0, "->", err, "eigenvalues", lam_hat, "population", lam)
    assert err0 > 0.5 and err < 0.25
    assert np.all(np.abs(np.sort(lam_hat)[::-1] - lam) < 0.3 * lam)
