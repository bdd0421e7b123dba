"""Several steps of the cluster path in one persistent launch (sgep_step_many): the same
sequence of minibatches gives the same players as one launch per step (sgep_step), across
launch boundaries and mixed with single steps, and one launch carries up to 64 steps.

Both runs apply Alg. 2's update with identical arithmetic; they differ only in the order in
which the clusters' float atomics land, which changes results in the last bits. Over tens of
steps those differences stay below 1e-4 relative (the bar of the other multi-step tests)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2206_04993_gb300 import Solver, sgep as S  # noqa: E402

KINDS = {"pca": S.SGEP_PCA, "cca": S.SGEP_CCA, "pls": S.SGEP_PLS}
CHAIN_TOL = 1e-4


def _rows(kind, dx, dy, n, seed):
    if kind == "pca":
        model = synth.planted_pca(dx, np.linspace(4, 1, min(8, dx)), seed=seed)
        return synth.draw_pca_rows(model, n, batch=seed), None
    model = synth.planted_cca(dx, dy, np.linspace(0.9, 0.3, max(1, min(8, dx, dy))), seed=seed)
    return synth.draw_rows(model, n, batch=seed)


def _solver(kind, dx, dy, k, dtype, b):
    return Solver(kind=KINDS[kind], d_x=dx, d_y=(0 if kind == "pca" else dy), k=k,
                  dtype=S.SGEP_BF16 if dtype == "bf16" else S.SGEP_F32, path=S.SGEP_PATH_CLUSTER,
                  eta0=0.1, gamma0=0.5, rho=1e-6, schedule=S.SGEP_SCHED_HOLD_HARMONIC, t_c=10, T=200,
                  eta_T=0.02, max_b=b)


def _dev(a, dtype):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return t.to(torch.bfloat16) if dtype == "bf16" else t


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kind,dx,dy,k,b", [("cca", 512, 512, 16, 1024), ("cca", 37, 29, 3, 101),
                                            ("pls", 64, 48, 5, 200), ("pca", 96, 0, 6, 128)])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_one_launch_matches_one_launch_per_step(kind, dx, dy, k, b, dtype):
    n = 40
    X, Y = _rows(kind, dx, dy, n * b, seed=3)
    Xd, Yd = _dev(X, dtype), (None if Y is None else _dev(Y, dtype))
    V0 = synth.random_unit_columns(dx + (0 if kind == "pca" else dy), k, seed=4).astype(np.float32)
    out = {}
    for mode in ("per_step", "many"):
        with _solver(kind, dx, dy, k, dtype, b) as s:
            s.set_V(V0)
            l0 = s.launches
            if mode == "many":
                s.step_many(Xd, Yd, b, n)
            else:
                for t in range(n):
                    s.step(Xd[t * b:(t + 1) * b], None if Yd is None else Yd[t * b:(t + 1) * b])
            launches = s.launches - l0
            out[mode] = (s.V(), s.S(), s.t, launches)
    (Vp, Sp, tp, lp), (Vm, Sm, tm, lm) = out["per_step"], out["many"]
    assert tp == tm == n
    assert lp == n and lm == 1, (lp, lm)
    assert _rel(Vm, Vp) < CHAIN_TOL and _rel(Sm, Sp) < CHAIN_TOL, (_rel(Vm, Vp), _rel(Sm, Sp))


def test_mixed_calls_across_launch_boundaries():
    """3 single steps, 70 steps in one call (a 64-step and a 6-step launch), 2 single steps and
    5 more in one call: the players match 80 single steps, and the step-size schedule (which
    changes every step) is applied to the right minibatch across every boundary."""
    dx, dy, k, b = 32, 32, 4, 256
    X, Y = _rows("cca", dx, dy, 80 * b, seed=8)
    Xd, Yd = _dev(X, "f32"), _dev(Y, "f32")
    V0 = synth.random_unit_columns(dx + dy, k, seed=9).astype(np.float32)

    def mb(t0, n):
        return Xd[t0 * b:(t0 + n) * b], Yd[t0 * b:(t0 + n) * b]

    with _solver("cca", dx, dy, k, "f32", b) as ref:
        ref.set_V(V0)
        for t in range(80):
            ref.step(*mb(t, 1))
        Vr, Sr = ref.V(), ref.S()
    with _solver("cca", dx, dy, k, "f32", b) as s:
        s.set_V(V0)
        t = 0
        for n, many in ((3, False), (70, True), (2, False), (5, True)):
            l0 = s.launches
            if many:
                s.step_many(*mb(t, n), b, n)
                assert s.launches - l0 == (n + 63) // 64
            else:
                for u in range(n):
                    s.step(*mb(t + u, 1))
            t += n
        assert s.t == 80
        Vm, Sm = s.V(), s.S()
    assert _rel(Vm, Vr) < CHAIN_TOL and _rel(Sm, Sr) < CHAIN_TOL, (_rel(Vm, Vr), _rel(Sm, Sr))


def test_multi_step_launch_tracks_the_oracle():
    """Twenty steps in one launch against the FP64 oracle run on the same minibatches."""
    from oracle import eg
    cfg = synth.config_c1()
    dx, k, b = 32, 4, 256
    idx = np.concatenate([synth.finite_dataset_indices(10_000, b, t) for t in range(1, 21)])
    X, Y = cfg["X"][idx].astype(np.float32), cfg["Y"][idx].astype(np.float32)
    V = synth.random_unit_columns(2 * dx, k, seed=0)
    Vr, Sr = V.copy(), V.copy()
    for t in range(20):
        Xt, Yt = X[t * b:(t + 1) * b], Y[t * b:(t + 1) * b]
        Vr, Sr = eg.eg_step(Vr, Sr, *eg.cca_ops(Xt, Yt), 0.2, 0.3, 1e-6)
    with Solver(kind=S.SGEP_CCA, d_x=dx, d_y=dx, k=k, path=S.SGEP_PATH_CLUSTER, eta0=0.2, gamma0=0.3,
                rho=1e-6, max_b=b) as s:
        s.set_V(V.astype(np.float32))
        l0 = s.launches
        s.step_many(_dev(X, "f32"), _dev(Y, "f32"), b, 20)
        assert s.launches - l0 == 1
        Vg, Sg = s.V(), s.S()
    assert _rel(Vg, Vr) < CHAIN_TOL and _rel(Sg, Sr) < CHAIN_TOL, (_rel(Vg, Vr), _rel(Sg, Sr))
