"""The allocation-free step (sgep_step_noalloc) against the handle-based step.

Callers that cannot allocate device memory (plugins handed fixed buffers by a
host application that owns the GPU's memory, services with a fixed device
footprint, loops where cudaMalloc's device-wide synchronisation is not
allowed) use this entry point with their own inputs and outputs; its
temporaries live in a fixed device array inside the library. Two calls in a
row must give what two sgep_step calls on a handle give, within the step
tolerance of the other GPU tests. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth
from paper_2206_04993_gb300 import sgep as S

STEP_TOL = 1e-5


def _cfg(**kw):
    return S.sgep_config_default(kind=S.SGEP_CCA, d_x=96, d_y=80, k=8, eta0=0.25, gamma0=0.4,
                                 rho=1e-4, path=S.SGEP_PATH_GENERIC, **kw)


def test_noalloc_rejects_shapes_beyond_the_fixed_scratch():
    cfg = _cfg()
    cfg.d_x, cfg.d_y, cfg.k = 200_000, 200_000, 8   # 3 d k floats alone exceed 4 MiB
    rc = S.lib().sgep_step_noalloc(ctypes.byref(cfg), 1, 1, 64, 1, 1, 1, 1, 1, None)
    assert rc == S.SGEP_EINVAL
    assert "scratch" in S.sgep_last_error()
    rc = S.lib().sgep_step_noalloc(ctypes.byref(_cfg()), None, None, 64, 1, 1, 1, 1, 1, None)
    assert rc == S.SGEP_EINVAL


@pytest.mark.gpu
def test_noalloc_step_matches_handle_step_twice():
    torch = pytest.importorskip("torch")
    from paper_2206_04993_gb300 import Solver
    model = synth.planted_cca(96, 80, np.linspace(0.9, 0.3, 8), seed=21)
    batches = [synth.draw_rows(model, 130, batch=i) for i in range(2)]
    V0 = synth.random_unit_columns(176, 8, seed=3).astype(np.float32)
    S0 = (0.8 * V0 + 0.05 * synth.random_unit_columns(176, 8, seed=4)).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731

    cfg = _cfg()
    stream = torch.cuda.current_stream()
    V_in, S_in = dev(V0), dev(S0)
    V_out, S_out = torch.empty_like(V_in), torch.empty_like(S_in)
    outs = []
    for t, (X, Y) in enumerate(batches, start=1):
        S.sgep_step_noalloc(cfg, dev(X), dev(Y), X.shape[0], V_in, S_in, V_out, S_out, t, stream)
        torch.cuda.synchronize()
        outs.append((V_out.cpu().numpy().copy(), S_out.cpu().numpy().copy()))
        V_in, S_in = V_out.clone(), S_out.clone()

    with Solver(kind=S.SGEP_CCA, d_x=96, d_y=80, k=8, eta0=0.25, gamma0=0.4, rho=1e-4,
                path=S.SGEP_PATH_GENERIC) as s:
        s.set_V(V0, S0)
        for t, (X, Y) in enumerate(batches):
            s.step(dev(X), dev(Y))
            Vh, Sh = s.V(), s.S()
            Vn, Sn = outs[t]
            assert np.linalg.norm(Vn - Vh) / np.linalg.norm(Vh) <= STEP_TOL
            assert np.linalg.norm(Sn - Sh) / np.linalg.norm(Sh) <= STEP_TOL
    # the second call really moved the state
    assert np.linalg.norm(outs[1][0] - outs[0][0]) > 1e-3


@pytest.mark.gpu
def test_noalloc_steps_match_the_oracle():
    """The same two allocation-free calls against two FP64 oracle steps of Alg. 2 on the same
    rows: whole-matrix and per-column errors of V and [Bv], two steps' worth of the step bar."""
    torch = pytest.importorskip("torch")
    from gpu_util import assert_within, col_errors, rel
    from oracle import eg
    model = synth.planted_cca(96, 80, np.linspace(0.9, 0.3, 8), seed=22)
    batches = [synth.draw_rows(model, 131, batch=i, dtype=np.float32) for i in range(2)]
    V0 = synth.random_unit_columns(176, 8, seed=5).astype(np.float32)
    S0 = (0.8 * V0 + 0.05 * synth.random_unit_columns(176, 8, seed=6)).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    cfg = _cfg()
    stream = torch.cuda.current_stream()
    V_in, S_in = dev(V0), dev(S0)
    V_out, S_out = torch.empty_like(V_in), torch.empty_like(S_in)
    Vr, Sr = V0.astype(np.float64), S0.astype(np.float64)
    for t, (X, Y) in enumerate(batches, start=1):
        S.sgep_step_noalloc(cfg, dev(X), dev(Y), X.shape[0], V_in, S_in, V_out, S_out, t, stream)
        torch.cuda.synchronize()
        V_in, S_in = V_out.clone(), S_out.clone()
        Vr, Sr = eg.eg_step(Vr, Sr, *eg.cca_ops(X, Y), 0.25, 0.4, 1e-4)
    Vg, Sg = V_out.cpu().numpy(), S_out.cpu().numpy()
    err = {"V": rel(Vg, Vr), "S": rel(Sg, Sr)}
    err["V_col"], err["V_elem"] = col_errors(Vg, Vr)
    err["S_col"], err["S_elem"] = col_errors(Sg, Sr)
    print(err)
    assert_within(err, 2 * STEP_TOL)
