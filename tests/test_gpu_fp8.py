"""FP8 e4m3 rows with per-row scales (precision form) on the GPU against the oracle,
which decodes the codes itself (oracle/fp8.py) and runs the FP64 step on the values."""
import numpy as np
import pytest

import synth
from gpu_util import STEP_TOL, oracle_ops, rel, to_device
from oracle import eg, fp8
from paper_2206_04993_gb300 import sgep as S

pytestmark = pytest.mark.gpu

KINDS = {"cca": S.SGEP_CCA, "pca": S.SGEP_PCA, "pls": S.SGEP_PLS}


def _dev(a, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _solver(kind, dx, dy, k, max_b, dtype=S.SGEP_FP8E4M3, **kw):
    from paper_2206_04993_gb300 import Solver
    return Solver(kind=KINDS[kind], d_x=dx, d_y=dy, k=k, max_b=max_b, dtype=dtype, debug=1, **kw)


@pytest.mark.parametrize("kind,dx,dy,k,b", [("cca", 64, 48, 6, 256), ("cca", 300, 212, 16, 500),
                                            ("pca", 257, 0, 9, 300), ("pls", 40, 40, 4, 128)],
                         ids=["cca", "cca_ragged", "pca", "pls"])
def test_fp8_step_matches_oracle(kind, dx, dy, k, b):
    import torch
    rng = np.random.default_rng(1)
    X = rng.standard_normal((b, dx)) * rng.uniform(0.1, 10.0, b)[:, None]
    Y = None if kind == "pca" else 0.5 * X[:, :dy] + rng.standard_normal((b, dy)) if dy <= dx else None
    cx, sx = synth.quantize_e4m3_rows(X)
    Xv = fp8.dequantize_rows(cx, sx)
    cy = sy = Yv = None
    if Y is not None:
        cy, sy = synth.quantize_e4m3_rows(Y)
        Yv = fp8.dequantize_rows(cy, sy)
    d = dx + dy
    V0 = synth.random_unit_columns(d, k, seed=2).astype(np.float32)
    S0 = (0.8 * V0 + 0.2 * synth.random_unit_columns(d, k, seed=3)).astype(np.float32)
    with _solver(kind, dx, dy, k, b, eta0=0.1, gamma0=0.4) as s:
        s.set_V(V0, S0)
        s.step(_dev(cx), None if cy is None else _dev(cy), b, sx=_dev(sx), sy=None if sy is None else _dev(sy))
        AVg, BVg = s.products()
        torch.cuda.synchronize()
        Vg, Sg = s.V(), s.S()
    Amv, Bmv = oracle_ops(kind, Xv, Yv, split=True, eps_B=0.0)
    V1, S1, parts = eg.eg_step(V0.astype(np.float64), S0.astype(np.float64), Amv, Bmv, 0.1, 0.4, 1e-6,
                               return_parts=True)
    errs = {"AV": rel(AVg, parts["AV"]), "V": rel(Vg, V1), "S": rel(Sg, S1)}
    if kind == "cca":
        errs["BV"] = rel(BVg, parts["BV"])
    for name, e in errs.items():
        assert e <= STEP_TOL, (name, e, errs)


def test_fp8_lda_steps_match_oracle():
    import torch
    from paper_2206_04993_gb300 import Solver
    d, k, C, b = 200, 4, 6, 256
    model = synth.planted_lda(d, n_classes=C, seed=7)
    V = synth.random_unit_columns(d, k, seed=8).astype(np.float32)
    sums, counts = np.zeros((C, d)), np.zeros(C)
    with Solver(kind=S.SGEP_LDA, d_x=d, d_y=0, k=k, n_classes=C, max_b=b, dtype=S.SGEP_FP8E4M3,
                eta0=0.05, gamma0=0.5, debug=1) as s:
        s.set_V(V)
        Vr, Sr = V.astype(np.float64), V.astype(np.float64)
        for t in range(3):
            X, lab = synth.draw_lda_rows(model, b, batch=t)
            cx, sx = synth.quantize_e4m3_rows(X)
            Xv = fp8.dequantize_rows(cx, sx)
            s.step(_dev(cx), None, b, labels=_dev(lab), sx=_dev(sx))
            torch.cuda.synchronize()
            sums, counts = eg.lda_stats_update(sums, counts, Xv, lab)
            mean, prior = eg.lda_state(sums, counts)
            V1, S1 = eg.eg_step(Vr, Sr, *eg.lda_ops(Xv, lab, mean, prior), 0.05, 0.5, 1e-6)
            assert rel(s.V(), V1) <= STEP_TOL and rel(s.S(), S1) <= STEP_TOL, t
            Vr, Sr = s.V().astype(np.float64), s.S().astype(np.float64)


def test_fp8_readout_and_rr_equal_the_dequantised_f32_rows():
    """The same values given as FP8 codes + scales and as FP32 rows give the same
    eigenvalue readout and the same Rayleigh-Ritz rotation."""
    import torch
    dx = dy = 96
    k, n = 5, 3000
    model = synth.planted_cca(dx, dy, np.linspace(0.9, 0.4, 8), sigma=0.5, seed=9)
    X, Y = synth.draw_rows(model, n, batch=3)
    cx, sx = synth.quantize_e4m3_rows(X)
    cy, sy = synth.quantize_e4m3_rows(Y)
    Xv, Yv = fp8.dequantize_rows(cx, sx).astype(np.float32), fp8.dequantize_rows(cy, sy).astype(np.float32)
    V0 = synth.random_unit_columns(dx + dy, k, seed=10).astype(np.float32)
    out = []
    for dtype in (S.SGEP_FP8E4M3, S.SGEP_F32):
        with _solver("cca", dx, dy, k, 1024, dtype=dtype, path=S.SGEP_PATH_GENERIC) as s:
            s.set_V(V0)
            if dtype == S.SGEP_FP8E4M3:
                a = (_dev(cx), _dev(cy))
                kw = {"sx": _dev(sx), "sy": _dev(sy)}
            else:
                a = (to_device(Xv, "f32"), to_device(Yv, "f32"))
                kw = {}
            lam = s.eigenvalues(*a, **kw)
            rr = s.rayleigh_ritz(*a, **kw)
            torch.cuda.synchronize()
            out.append((lam, rr, s.V()))
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-5)
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-5)
    assert rel(out[0][2], out[1][2]) < 1e-5


def test_row_scale_arguments_are_checked():
    import torch
    X = np.zeros((8, 16), dtype=np.uint8)
    sc = np.ones(8, dtype=np.float32)
    with _solver("pca", 16, 0, 2, 8) as s:
        with pytest.raises(S.SgepError) as ei:
            s.step(_dev(X), None, 8)  # FP8 rows without their scales
        assert ei.value.status == S.SGEP_EINVAL
        with pytest.raises(S.SgepError) as ei:
            s.step(_dev(X), None, 8, sx=_dev(sc), sy=_dev(sc))  # a scale for a view that does not exist
        assert ei.value.status == S.SGEP_EINVAL
    with _solver("pca", 16, 0, 2, 8, dtype=S.SGEP_F32) as s:
        with pytest.raises(S.SgepError) as ei:
            s.step(to_device(np.zeros((8, 16)), "f32"), None, 8, sx=_dev(sc))  # scales for FP32 rows
        assert ei.value.status == S.SGEP_EINVAL
    torch.cuda.synchronize()
