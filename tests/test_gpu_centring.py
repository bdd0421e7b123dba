"""GPU parity of running-mean centring (App. H.2.2 "mean estimates are learned"; the pencils
of Sec. 1 assume zero-mean data) against the FP64 oracle, on rows with a large offset."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import synth  # noqa: E402
from gpu_util import bf16_round, rel, to_device  # noqa: E402
from oracle import eg  # noqa: E402
from paper_2206_04993_gb300 import Solver  # noqa: E402
from paper_2206_04993_gb300 import sgep as S  # noqa: E402

TOL = 1e-5


def _rows(model, b, batch, off_x, off_y, dtype):
    X, Y = synth.draw_rows(model, b, batch=batch)
    X, Y = X + off_x, Y + off_y
    if dtype == "bf16":
        return bf16_round(X), bf16_round(Y)
    return np.asarray(X, np.float32), np.asarray(Y, np.float32)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_centred_steps_match_oracle(dtype):
    model = synth.planted_cca(32, 32, np.linspace(0.9, 0.3, 8), seed=6)
    off_x, off_y = np.linspace(-4.0, 4.0, 32), np.linspace(3.0, -1.0, 32)
    V0 = synth.random_unit_columns(64, 4, seed=3).astype(np.float32)
    Vr, Sr = V0.astype(np.float64), V0.astype(np.float64)
    sums, n = np.zeros(64), 0.0
    with Solver(kind=S.SGEP_CCA, d_x=32, d_y=32, k=4, dtype=S.SGEP_BF16 if dtype == "bf16" else S.SGEP_F32,
                eta0=0.2, gamma0=0.4, rho=1e-4, center=1, max_b=256) as s:
        assert s.path == S.SGEP_PATH_GENERIC
        s.set_V(V0)
        for t in range(3):
            X, Y = _rows(model, 256, 50 + t, off_x, off_y, dtype)
            s.step(to_device(X, dtype), to_device(Y, dtype))
            sums, n, mean = eg.running_mean_update(sums, n, np.hstack([X, Y]))
            Xc = np.asarray(X, np.float64) - mean[:32]
            Yc = np.asarray(Y, np.float64) - mean[32:]
            Vr, Sr = eg.eg_step(Vr, Sr, *eg.cca_ops(Xc, Yc), 0.2, 0.4, 1e-4)
            ev, es = rel(s.V(), Vr), rel(s.S(), Sr)
            assert ev <= TOL and es <= TOL, (t, ev, es)


def test_centring_removes_a_constant_offset():
    """Two handles fed the same rows with and without a constant offset move the same way."""
    model = synth.planted_cca(32, 32, np.linspace(0.9, 0.3, 8), seed=8)
    off_x, off_y = np.full(32, 7.0), np.linspace(-2.0, 2.0, 32)
    kw = dict(kind=S.SGEP_CCA, d_x=32, d_y=32, k=4, eta0=0.2, gamma0=0.4, rho=1e-4, center=1, max_b=256, seed=4)
    with Solver(**kw) as a, Solver(**kw) as b:
        for t in range(20):
            X, Y = synth.draw_rows(model, 256, batch=70 + t)
            X0, Y0 = np.asarray(X, np.float32), np.asarray(Y, np.float32)
            a.step(to_device(X0, "f32"), to_device(Y0, "f32"))
            b.step(to_device(np.asarray(X + off_x, np.float32), "f32"),
                   to_device(np.asarray(Y + off_y, np.float32), "f32"))
        assert rel(b.V(), a.V().astype(np.float64)) < 1e-4


def test_centring_state_round_trip():
    model = synth.planted_cca(32, 32, np.linspace(0.9, 0.3, 8), seed=9)
    rows = [_rows(model, 256, 90 + t, 3.0, -2.0, "f32") for t in range(5)]
    dev = [(to_device(X, "f32"), to_device(Y, "f32")) for X, Y in rows]
    kw = dict(kind=S.SGEP_CCA, d_x=32, d_y=32, k=4, eta0=0.2, gamma0=0.4, rho=1e-4, center=1, max_b=256, seed=2)
    with Solver(**kw) as a:
        for X, Y in dev[:3]:
            a.step(X, Y)
        blob = a.state()
        for X, Y in dev[3:]:
            a.step(X, Y)
        Va = a.V()
    with Solver(**kw) as b:
        b.load_state(blob)
        for X, Y in dev[3:]:
            b.step(X, Y)
        assert rel(b.V(), Va.astype(np.float64)) < 1e-6


def test_centring_config_checks():
    for kw in ({"center": 2}, {"center": 1, "kind": S.SGEP_LDA, "n_classes": 3, "d_y": 0}):
        args = dict(kind=S.SGEP_CCA, d_x=32, d_y=32, k=4)
        args.update(kw)
        with pytest.raises(S.SgepError) as ei:
            Solver(**args)
        assert ei.value.status == S.SGEP_EINVAL
    with pytest.raises(S.SgepError) as ei:
        Solver(kind=S.SGEP_CCA, d_x=512, d_y=512, k=16, center=1, dtype=S.SGEP_BF16, path=S.SGEP_PATH_TC)
    assert ei.value.status == S.SGEP_ENOTSUP
