"""Periodic Rayleigh-Ritz correction (precision form) against the oracle: Alg. 2 steps with the
Ritz step of App. A (Prop. "Similar matrices") applied on an evaluation batch after every
`every` steps, on the generic FP32 path and on the streamed tensor-core path (where the
multi-step launches are split at the corrections)."""
import numpy as np
import pytest

import synth
from gpu_util import bf16_round, rel
from oracle import eg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2206_04993_gb300 import Solver, sgep as S  # noqa: E402


def _match_up_to_sign(A, B):
    """A with each column's sign chosen to agree with B (the update is sign-equivariant per player)."""
    s = np.sign(np.sum(A * B, axis=0))
    s[s == 0] = 1
    return A * s[None, :], s


def _oracle(X, Y, Xe, Ye, V0, S0, b, n, every, eta, gamma, rho):
    V, Sv = V0.astype(np.float64), S0.astype(np.float64)
    Ae, Be = eg.cca_ops(Xe, Ye, split=False)  # the evaluation batch estimates A and B on all rows
    for t in range(1, n + 1):
        r = slice((t - 1) * b, t * b)
        V, Sv = eg.eg_step(V, Sv, *eg.cca_ops(X[r], Y[r]), eta, gamma, rho)
        if t % every == 0:
            V, Sv, _ = eg.rayleigh_ritz(V, Sv, Ae, Be)
    return V, Sv


def _check(Vg, Sg, Vr, Sr, tol):
    Vs, sg = _match_up_to_sign(Vg.astype(np.float64), Vr)
    ev, es = rel(Vs, Vr), rel(Sg * sg[None, :], Sr)
    print({"V": ev, "S": es})
    assert ev < tol and es < tol


def test_periodic_rr_generic_path_matches_oracle():
    dx, dy, k, b, n, every = 40, 24, 5, 256, 7, 3
    model = synth.planted_cca(dx, dy, np.linspace(0.9, 0.4, 8), seed=13)
    X, Y = synth.draw_rows(model, b * n, batch=2, dtype=np.float32)
    Xe, Ye = synth.draw_rows(model, 900, batch=3, dtype=np.float32)
    V0 = synth.random_unit_columns(dx + dy, k, seed=8).astype(np.float32)
    S0 = (0.8 * V0 + 0.05 * synth.random_unit_columns(dx + dy, k, seed=9)).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    Xed, Yed = torch.from_numpy(Xe).cuda(), torch.from_numpy(Ye).cuda()
    with Solver(kind=S.SGEP_CCA, d_x=dx, d_y=dy, k=k, path=S.SGEP_PATH_GENERIC, eta0=0.3, gamma0=0.4, rho=1e-3,
                max_b=b) as s:
        s.set_V(V0, S0)
        s.set_rr_every(every, Xed, Yed)
        for t in range(n):
            s.step(Xd[t * b:(t + 1) * b], Yd[t * b:(t + 1) * b])
        s.sync()
        Vg, Sg = s.V(), s.S()
        assert s.t == n
    Vr, Sr = _oracle(X.astype(np.float64), Y.astype(np.float64), Xe.astype(np.float64), Ye.astype(np.float64),
                     V0, S0, b, n, every, 0.3, 0.4, 1e-3)
    _check(Vg, Sg, Vr, Sr, n * 1e-5)


def test_periodic_rr_streamed_tc_path_matches_oracle():
    dx, k, b, n, every = 512, 8, 256, 5, 2
    model = synth.planted_cca(dx, dx, np.linspace(0.9, 0.4, 8), seed=14)
    X, Y = synth.draw_rows(model, b * n, batch=4, dtype=np.float32)
    Xe, Ye = synth.draw_rows(model, 1024, batch=5, dtype=np.float32)
    Xv, Yv, Xev, Yev = (bf16_round(a) for a in (X, Y, Xe, Ye))
    V0 = synth.random_unit_columns(2 * dx, k, seed=10).astype(np.float32)
    S0 = (0.8 * V0 + 0.05 * synth.random_unit_columns(2 * dx, k, seed=11)).astype(np.float32)
    to_bf16 = lambda a: torch.from_numpy(a).cuda().to(torch.bfloat16)  # noqa: E731
    Xd, Yd, Xed, Yed = to_bf16(X), to_bf16(Y), to_bf16(Xe), to_bf16(Ye)
    with Solver(kind=S.SGEP_CCA, d_x=dx, d_y=dx, k=k, dtype=S.SGEP_BF16, path=S.SGEP_PATH_TC, eta0=0.3,
                gamma0=0.4, rho=1e-3, max_b=b) as s:
        s.set_V(V0, S0)
        s.set_rr_every(every, Xed, Yed)
        s.step_many(Xd, Yd, b, n)  # launches of 2, 2 and 1 steps, corrections after steps 2 and 4
        s.sync()
        Vg, Sg = s.V(), s.S()
        assert s.t == n
        s.set_rr_every(0)
    Vr, Sr = _oracle(Xv.astype(np.float64), Yv.astype(np.float64), Xev.astype(np.float64), Yev.astype(np.float64),
                     V0, S0, b, n, every, 0.3, 0.4, 1e-3)
    _check(Vg, Sg, Vr, Sr, n * 5e-5)


def test_set_rr_every_rejects_bad_arguments():
    with Solver(kind=S.SGEP_CCA, d_x=8, d_y=8, k=2, path=S.SGEP_PATH_GENERIC, max_b=64) as s:
        with pytest.raises(S.SgepError):
            S.sgep_set_rr_every(s.h, -1)
        with pytest.raises(S.SgepError):
            S.sgep_set_rr_every(s.h, 5)  # no evaluation rows
        s.set_rr_every(0)  # removing an absent schedule is fine
