"""Batching form: many uneven instances (CCA, PCA, PLS, LDA; FP32, BF16, FP8 rows)
advanced by one batched launch per step, against the same handles stepped one by one
and against the oracle; launch modes, graph replay, the autotuner, argument errors."""
import numpy as np
import pytest

import synth
from gpu_util import STEP_TOL, bf16_round, oracle_ops, rel, to_device
from oracle import eg, fp8
from paper_2206_04993_gb300 import sgep as S

pytestmark = pytest.mark.gpu

# (kind, d_x, d_y, k, b, dtype, n_classes)
SPECS = [
    ("cca", 64, 64, 4, 128, "f32", 0),
    ("cca", 300, 212, 16, 256, "bf16", 0),
    ("pca", 257, 0, 9, 200, "f32", 0),
    ("pls", 40, 40, 3, 64, "f32", 0),
    ("lda", 200, 0, 4, 256, "f32", 6),
    ("lda", 96, 0, 2, 128, "bf16", 3),
    ("cca", 128, 128, 8, 256, "fp8", 0),
]
KIND = {"cca": S.SGEP_CCA, "pca": S.SGEP_PCA, "pls": S.SGEP_PLS, "lda": S.SGEP_LDA}
DT = {"f32": S.SGEP_F32, "bf16": S.SGEP_BF16, "fp8": S.SGEP_FP8E4M3}


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _make(spec, seed):
    from paper_2206_04993_gb300 import Solver
    kind, dx, dy, k, b, dt, C = spec
    s = Solver(kind=KIND[kind], d_x=dx, d_y=dy, k=k, max_b=b, dtype=DT[dt], n_classes=C, path=S.SGEP_PATH_GENERIC,
               eta0=0.1, gamma0=0.4, seed=seed)
    return s


def _rows(spec, t, seed):
    """Device rows of step t for one instance: dict with X, Y, labels, sx, sy and host values."""
    kind, dx, dy, k, b, dt, C = spec
    rng = np.random.default_rng(1000 * seed + t)
    out = {"labels": None, "sx": None, "sy": None, "Y": None, "Yv": None, "lab": None}
    if kind == "lda":
        model = synth.planted_lda(dx, n_classes=C, seed=seed)
        X, lab = synth.draw_lda_rows(model, b, batch=t)
        out["lab"] = lab
        out["labels"] = _dev(lab)
        Y = None
    else:
        X = rng.standard_normal((b, dx))
        X[:, :2] *= 3.0
        Y = None if kind == "pca" else 0.6 * X[:, :dy] + rng.standard_normal((b, dy)) if dy <= dx else \
            rng.standard_normal((b, dy))
    for name, M in (("X", X), ("Y", Y)):
        if M is None:
            continue
        if dt == "fp8":
            codes, sc = synth.quantize_e4m3_rows(M)
            out[name] = _dev(codes)
            out["s" + name.lower()] = _dev(sc)
            out[name + "v"] = fp8.dequantize_rows(codes, sc)
        else:
            v = bf16_round(M) if dt == "bf16" else M.astype(np.float32)
            out[name] = to_device(v, dt)
            out[name + "v"] = v
    return out


def _run(mode, graph, nsteps=3):
    import torch
    from paper_2206_04993_gb300 import Batch
    solo = [_make(sp, i) for i, sp in enumerate(SPECS)]
    grouped = [_make(sp, i) for i, sp in enumerate(SPECS)]
    try:
        with Batch(grouped) as bt:
            bt.configure(mode=mode, use_graph=int(graph))
            for t in range(nsteps):
                rows = [_rows(sp, t, i) for i, sp in enumerate(SPECS)]
                for s, r, sp in zip(solo, rows, SPECS):
                    s.step(r["X"], r["Y"], sp[4], labels=r["labels"], sx=r["sx"], sy=r["sy"])
                bt.step([r["X"] for r in rows], [r["Y"] for r in rows], [sp[4] for sp in SPECS],
                        labels=[r["labels"] for r in rows], sx=[r["sx"] for r in rows], sy=[r["sy"] for r in rows])
            bt.sync()
            launches = bt.launches()
            torch.cuda.synchronize()
            errs = [(rel(g.V(), s.V()), rel(g.S(), s.S())) for g, s in zip(grouped, solo)]
            steps = [g.t for g in grouped]
    finally:
        for s in solo + grouped:
            s.close()
    return errs, launches, steps


@pytest.mark.parametrize("mode,graph", [(0, False), (1, False), (0, True), (1, True)],
                         ids=["persistent", "per_phase", "persistent_graph", "per_phase_graph"])
def test_batch_equals_individual_steps(mode, graph):
    errs, launches, steps = _run(mode, graph)
    for i, (ev, es) in enumerate(errs):
        assert ev <= STEP_TOL and es <= STEP_TOL, (SPECS[i], ev, es)
    assert steps == [3] * len(SPECS)
    assert launches == (3 if mode == 0 else 3 * 8)


def test_batch_step_matches_oracle():
    """One batched step of two instances against the oracle directly."""
    import torch
    from paper_2206_04993_gb300 import Batch
    specs = [SPECS[1], SPECS[4]]
    ss = [_make(sp, i) for i, sp in enumerate(specs)]
    V0 = [s.V().astype(np.float64) for s in ss]
    rows = [_rows(sp, 0, i) for i, sp in enumerate(specs)]
    with Batch(ss) as bt:
        bt.step([r["X"] for r in rows], [r["Y"] for r in rows], [sp[4] for sp in specs],
                labels=[r["labels"] for r in rows])
        bt.sync()
    torch.cuda.synchronize()
    # CCA instance (BF16 rows)
    Amv, Bmv = oracle_ops("cca", rows[0]["Xv"], rows[0]["Yv"], split=True, eps_B=0.0)
    V1, S1 = eg.eg_step(V0[0], V0[0], Amv, Bmv, 0.1, 0.4, 1e-6)
    assert rel(ss[0].V(), V1) <= STEP_TOL and rel(ss[0].S(), S1) <= STEP_TOL
    # LDA instance
    C = specs[1][6]
    sums, counts = eg.lda_stats_update(np.zeros((C, specs[1][1])), np.zeros(C), rows[1]["Xv"], rows[1]["lab"])
    mean, prior = eg.lda_state(sums, counts)
    V1, S1 = eg.eg_step(V0[1], V0[1], *eg.lda_ops(rows[1]["Xv"], rows[1]["lab"], mean, prior), 0.1, 0.4, 1e-6)
    assert rel(ss[1].V(), V1) <= STEP_TOL and rel(ss[1].S(), S1) <= STEP_TOL
    for s in ss:
        s.close()


def test_batch_autotune_restores_state_and_caches():
    import torch
    from paper_2206_04993_gb300 import Batch
    ss = [_make(sp, i) for i, sp in enumerate(SPECS)]
    rows = [_rows(sp, 0, i) for i, sp in enumerate(SPECS)]
    args = dict(Ys=[r["Y"] for r in rows], rows=[sp[4] for sp in SPECS], labels=[r["labels"] for r in rows],
                sx=[r["sx"] for r in rows], sy=[r["sy"] for r in rows])
    V0 = [s.V() for s in ss]
    with Batch(ss) as bt:
        cfg = bt.autotune([r["X"] for r in rows], reps=2, **args)
        assert cfg[0] in (0, 1) and cfg[2] in (256, 512, 1024) and cfg[3] in (64, 128, 256)
        assert bt.config() == cfg
        for s, v in zip(ss, V0):
            np.testing.assert_array_equal(s.V(), v)
            assert s.t == 0
        assert bt.autotune([r["X"] for r in rows], reps=2, **args) == cfg  # cached
        bt.step([r["X"] for r in rows], **args)
        bt.sync()
    torch.cuda.synchronize()
    for s in ss:
        assert s.t == 1
        s.close()


def test_batch_argument_errors():
    from paper_2206_04993_gb300 import Batch, Solver
    a = _make(SPECS[0], 0)
    lda = _make(SPECS[4], 1)
    cl = Solver(kind=S.SGEP_CCA, d_x=64, d_y=64, k=4, max_b=128)  # auto path: not generic
    with pytest.raises(S.SgepError) as ei:
        Batch([a, a])
    assert ei.value.status == S.SGEP_EINVAL
    if cl.path != S.SGEP_PATH_GENERIC:
        with pytest.raises(S.SgepError) as ei:
            Batch([a, cl])
        assert ei.value.status == S.SGEP_EINVAL
    r0, r1 = _rows(SPECS[0], 0, 0), _rows(SPECS[4], 0, 1)
    with Batch([a, lda]) as bt:
        with pytest.raises(S.SgepError) as ei:  # LDA instance without labels
            bt.step([r0["X"], r1["X"]], [r0["Y"], None], [128, 256])
        assert ei.value.status == S.SGEP_EINVAL
        with pytest.raises(S.SgepError) as ei:  # rows beyond max_b
            bt.step([r0["X"], r1["X"]], [r0["Y"], None], [129, 256], labels=[None, r1["labels"]])
        assert ei.value.status == S.SGEP_EINVAL
    for s in (a, lda, cl):
        s.close()
