"""Rayleigh-Ritz correction on the GPU against the oracle (FP64 k x k solve on the device)."""
import numpy as np
import pytest

import synth
from gpu_util import bf16_round, oracle_ops, rel, to_device
from oracle import eg, gep
from paper_2206_04993_gb300 import sgep as S

pytestmark = pytest.mark.gpu

KINDS = {"cca": S.SGEP_CCA, "pca": S.SGEP_PCA, "pls": S.SGEP_PLS}


def _solver(kind, dx, dy, k, max_b, **kw):
    from paper_2206_04993_gb300 import Solver
    return Solver(kind=KINDS[kind], d_x=dx, d_y=dy, k=k, max_b=max_b, path=S.SGEP_PATH_GENERIC, **kw)


def _match_up_to_sign(A, B):
    s = np.sign(np.sum(A * B, axis=0))
    s[s == 0] = 1
    return A * s[None, :]


def _check(Vg, Sg, lamg, Vr, Sr, lamr, tol=2e-5):
    np.testing.assert_allclose(lamg, lamr, rtol=tol, atol=tol * np.abs(lamr).max())
    assert rel(_match_up_to_sign(Vg, Vr), Vr) < tol
    sg = np.sign(np.sum(Vg * Vr, axis=0))
    assert rel(Sg * sg[None, :], Sr) < tol


@pytest.mark.parametrize("kind,dx,dy,k,n", [("cca", 40, 24, 5, 700), ("pca", 96, 0, 7, 500),
                                             ("pls", 30, 30, 4, 300), ("cca", 300, 212, 16, 5000)],
                         ids=["cca", "pca", "pls", "cca_chunks"])
def test_rr_matches_oracle(kind, dx, dy, k, n):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((n, dx)).astype(np.float32)
    X[:, :3] *= 3.0
    Y = None if kind == "pca" else (0.5 * X[:, :dy] if dy <= dx else rng.standard_normal((n, dy))).astype(np.float32)
    if Y is not None:
        Y = Y + rng.standard_normal(Y.shape).astype(np.float32)
    d = dx + dy
    V0 = synth.random_unit_columns(d, k, seed=4).astype(np.float32)
    S0 = (0.7 * V0 + 0.3 * synth.random_unit_columns(d, k, seed=5)).astype(np.float32)
    with _solver(kind, dx, dy, k, max_b=1024) as s:
        s.set_V(V0, S0)
        lamg = s.rayleigh_ritz(to_device(X, "f32"), None if Y is None else to_device(Y, "f32"))
        Vg, Sg = s.V(), s.S()
    Amv, Bmv = oracle_ops(kind, X, Y, split=False, eps_B=0.0)
    Vr, Sr, lamr = eg.rayleigh_ritz(V0.astype(np.float64), S0.astype(np.float64), Amv, Bmv)
    _check(Vg, Sg, lamg, Vr, Sr, lamr)


def test_rr_lda_matches_oracle():
    import torch
    d, k, C, b = 64, 3, 5, 256
    model = synth.planted_lda(d, n_classes=C, seed=6)
    with pytest.importorskip("paper_2206_04993_gb300").Solver(kind=S.SGEP_LDA, d_x=d, d_y=0, k=k, n_classes=C,
                                                             max_b=b) as s:
        sums, counts = np.zeros((C, d)), np.zeros(C)
        for t in range(3):
            X, lab = synth.draw_lda_rows(model, b, batch=t)
            s.step(to_device(X, "f32"), None, b, labels=torch.from_numpy(lab).cuda())
            sums, counts = eg.lda_stats_update(sums, counts, X.astype(np.float32), lab)
        V0, S0 = s.V(), s.S()
        Xe, le = synth.draw_lda_rows(model, 2000, batch=50)
        lamg = s.rayleigh_ritz(to_device(Xe, "f32"), None, labels=torch.from_numpy(le).cuda())
        Vg, Sg = s.V(), s.S()
    mean, prior = eg.lda_state(sums, counts)
    Amv, Bmv = eg.lda_ops(Xe.astype(np.float32), le, mean, prior, split=False)
    Vr, Sr, lamr = eg.rayleigh_ritz(V0.astype(np.float64), S0.astype(np.float64), Amv, Bmv)
    _check(Vg, Sg, lamg, Vr, Sr, lamr, tol=1e-4)


def test_rr_improves_players_of_a_noisy_bf16_run():
    """After BF16 steps the span is close but the individual players are not: the correction
    brings each v_i to the planted canonical direction (the span error is unchanged)."""
    import torch
    cfg = synth.config_c2()
    model = cfg["model"]
    k, b = 8, 1024
    lam_t, Vt = gep.cca_truth_planted(model, k)
    Bop = lambda U: gep.cca_B_apply(model, U)  # noqa: E731
    X, Y = synth.draw_rows(model, b * 64, batch=11, dtype=np.float32)
    Xd, Yd = to_device(bf16_round(X), "bf16"), to_device(bf16_round(Y), "bf16")
    with _solver("cca", 512, 512, k, b, dtype=S.SGEP_BF16, eta0=0.2, gamma0=0.3) as s:
        s.step_many(Xd, Yd, b, 64)
        torch.cuda.synchronize()
        V1 = s.V().astype(np.float64)
        Xe, Ye = synth.draw_rows(model, 20000, batch=12, dtype=np.float32)
        s.rayleigh_ritz(to_device(Xe, "bf16"), to_device(Ye, "bf16"))
        V2 = s.V().astype(np.float64)
    span1 = gep.subspace_error(Vt, V1, Bop)
    span2 = gep.subspace_error(Vt, V2, Bop)
    assert abs(span2 - span1) < 1e-3 + 0.02 * span1

    def per_player(V):
        return float(np.mean(1.0 - np.abs(np.sum(V * Vt, axis=0)) / np.linalg.norm(V, axis=0)))
    assert per_player(V2) < per_player(V1), (per_player(V1), per_player(V2))


def test_rr_rejects_dependent_players():
    import torch
    d, k = 32, 3
    V0 = synth.random_unit_columns(d, k, seed=1).astype(np.float32)
    V0[:, 2] = V0[:, 1]  # two identical players: V^T B V is singular
    X = np.random.default_rng(0).standard_normal((200, d)).astype(np.float32)
    with _solver("pca", d, 0, k, 256) as s:
        s.set_V(V0)
        with pytest.raises(S.SgepError) as ei:
            s.rayleigh_ritz(to_device(X, "f32"))
        assert ei.value.status == S.SGEP_ENONFINITE
        np.testing.assert_array_equal(s.V(), V0)  # left unchanged
        torch.cuda.synchronize()
