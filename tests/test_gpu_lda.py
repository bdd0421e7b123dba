"""LDA on the GPU (generic path) against the oracle: running class statistics, the
between-class products from the class means, the within-class products of the
centred B rows, several consecutive steps, errors and state."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import STEP_TOL, bf16_round, rel, to_device
from oracle import eg, gep
from paper_2206_04993_gb300 import sgep as S

pytestmark = pytest.mark.gpu


def _solver(d, k, C, max_b, dtype="f32", **kw):
    from paper_2206_04993_gb300 import Solver
    kw.setdefault("eta0", 0.2)
    kw.setdefault("gamma0", 0.5)
    kw.setdefault("rho", 1e-6)
    return Solver(kind=S.SGEP_LDA, d_x=d, d_y=0, k=k, n_classes=C, max_b=max_b, debug=1,
                  dtype=S.SGEP_BF16 if dtype == "bf16" else S.SGEP_F32, **kw)


def _labels_dev(lab):
    import torch
    return torch.from_numpy(np.ascontiguousarray(lab, dtype=np.int32)).cuda()


def _run_steps(d, k, C, b, nsteps, dtype="f32", split=True, seed=0):
    """nsteps library steps and oracle steps from the same state; per-step relative errors."""
    import torch
    model = synth.planted_lda(d, n_classes=C, seed=seed)
    V = synth.random_unit_columns(d, k, seed=seed + 1).astype(np.float32)
    Sx = (0.9 * V + 0.1 * synth.random_unit_columns(d, k, seed=seed + 2)).astype(np.float32)
    sums, counts = np.zeros((C, d)), np.zeros(C)
    errs = []
    with _solver(d, k, C, b, dtype, split_AB=int(split)) as s:
        s.set_V(V, Sx)
        Vr, Sr = V.astype(np.float64), Sx.astype(np.float64)
        for t in range(nsteps):
            X, lab = synth.draw_lda_rows(model, b, batch=t)
            Xv = bf16_round(X) if dtype == "bf16" else X.astype(np.float32)
            s.step(to_device(Xv, dtype), None, b, labels=_labels_dev(lab))
            AVg, BVg = s.products()
            torch.cuda.synchronize()
            sums, counts = eg.lda_stats_update(sums, counts, Xv, lab)
            mean, prior = eg.lda_state(sums, counts)
            Amv, Bmv = eg.lda_ops(Xv, lab, mean, prior, split=split)
            V1, S1, parts = eg.eg_step(Vr, Sr, Amv, Bmv, 0.2, 0.5, 1e-6, return_parts=True)
            errs.append({"AV": rel(AVg, parts["AV"]), "BV": rel(BVg, parts["BV"]),
                         "V": rel(s.V(), V1), "S": rel(s.S(), S1)})
            # continue both from the library's state so that errors do not compound
            Vr, Sr = s.V().astype(np.float64), s.S().astype(np.float64)
    return errs


@pytest.mark.parametrize("d,k,C,b", [(64, 3, 4, 128), (300, 9, 10, 250), (1000, 16, 10, 512)],
                         ids=["d64", "d300_ragged", "d1000"])
def test_lda_steps_match_oracle(d, k, C, b):
    for t, e in enumerate(_run_steps(d, k, C, b, 4)):
        for name, v in e.items():
            assert v <= STEP_TOL, (t, name, v, e)


def test_lda_unsplit_batch():
    for e in _run_steps(200, 4, 5, 256, 3, split=False, seed=3):
        for name, v in e.items():
            assert v <= STEP_TOL, (name, v, e)


@pytest.mark.parametrize("d", [512, 301, 250], ids=["d512", "d301_odd", "d250_even"])
def test_lda_bf16_rows(d):
    """BF16 rows: 16-byte staging (d a multiple of 8), or the aligned value pairs holding each
    thread's values (odd d, and even d that is not a multiple of 8)."""
    for e in _run_steps(d, 8, 10, 256, 3, dtype="bf16", seed=5):
        for name, v in e.items():
            assert v <= STEP_TOL, (name, v, e)


def test_lda_bad_label_is_reported():
    import torch
    d, k, C, b = 32, 2, 3, 64
    X, lab = synth.draw_lda_rows(synth.planted_lda(d, n_classes=C, seed=1), b, batch=0)
    lab = lab.copy()
    lab[7] = C  # outside [0, C)
    with _solver(d, k, C, b) as s:
        s.step(to_device(X, "f32"), None, b, labels=_labels_dev(lab))
        with pytest.raises(S.SgepError) as ei:
            s.sync()
        assert ei.value.status == S.SGEP_EINVAL
        torch.cuda.synchronize()


def test_lda_requires_labels():
    d, k, C, b = 32, 2, 3, 64
    X, _ = synth.draw_lda_rows(synth.planted_lda(d, n_classes=C, seed=1), b, batch=0)
    with _solver(d, k, C, b) as s:
        with pytest.raises(S.SgepError) as ei:
            s.step(to_device(X, "f32"), None, b)
        assert ei.value.status == S.SGEP_EINVAL


def test_lda_state_roundtrip_keeps_class_statistics():
    import torch
    d, k, C, b = 48, 3, 4, 128
    model = synth.planted_lda(d, n_classes=C, seed=2)
    batches = [synth.draw_lda_rows(model, b, batch=t) for t in range(4)]
    with _solver(d, k, C, b) as s1, _solver(d, k, C, b) as s2:
        for X, lab in batches[:3]:
            s1.step(to_device(X, "f32"), None, b, labels=_labels_dev(lab))
        s2.load_state(s1.state())
        X, lab = batches[3]
        for s in (s1, s2):
            s.step(to_device(X, "f32"), None, b, labels=_labels_dev(lab))
        torch.cuda.synchronize()
        assert rel(s2.V(), s1.V()) < 1e-6 and rel(s2.S(), s1.S()) < 1e-6


def test_lda_converges_to_population_solution():
    """Planted Gaussian classes: the top generalized eigenvectors of the population
    between/within-class pencil are found, and the readout gives their eigenvalues."""
    import torch
    d, k, C, b = 32, 3, 5, 1024
    model = synth.planted_lda(d, n_classes=C, sigma_b=1.0, seed=4)
    A, B = gep.lda_population_AB(model)
    lam, Vt = gep.gep_topk(A, B, k)
    rows = [synth.draw_lda_rows(model, b, batch=t) for t in range(100)]
    Xall = to_device(np.concatenate([r[0] for r in rows]), "f32")
    Lall = _labels_dev(np.concatenate([r[1] for r in rows]))
    with _solver(d, k, C, b, eta0=0.05, gamma0=0.3, schedule=S.SGEP_SCHED_HOLD_HARMONIC, t_c=100, T=3000,
                 eta_T=0.005) as s:
        for rep in range(30):
            s.step_many(Xall, None, b, 100, labels=Lall)
        torch.cuda.synchronize()
        err = gep.subspace_error(Vt, s.V().astype(np.float64), B)
        Xe, le = synth.draw_lda_rows(model, 20000, batch=999)
        lam_hat = s.eigenvalues(to_device(Xe, "f32"), None, labels=_labels_dev(le))
    assert err < 2e-2, err
    np.testing.assert_allclose(lam_hat, lam, rtol=0.1)
