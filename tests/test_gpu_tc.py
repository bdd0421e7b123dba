"""GPU tests of the tensor-core building blocks and the tensor-core path."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2206_04993_gb300 import sgep as S  # noqa: E402


def test_tcgen05_kmajor_product():
    """TMA (128-byte swizzle) + tcgen05.mma BF16 -> FP32 + tcgen05.ld, A K-major."""
    assert S.sgep_tc_selftest(0) < 1e-6


def test_tcgen05_mnmajor_product():
    """The same product with A read transposed (MN-major) from a row-major tile."""
    errs = [S.sgep_tc_selftest(1), S.sgep_tc_selftest(2)]
    print("MN-major self-test errors (LBO=group stride, swapped):", errs)
    assert errs[0] < 1e-6


import synth  # noqa: E402
from gpu_util import step_errors  # noqa: E402

# The tensor-core path multiplies BF16 minibatch values by BF16 (hi, lo) pairs of V and of
# the row projections; a pair carries about 16 significant bits, so each product term has a
# relative error near 2^-17 before FP32 accumulation. The step parity bar for this path is
# therefore 5e-5 (relative, same metric as the FP32 path's 1e-5).
TC_TOL = 5e-5


def _tc_solver(dx, k, **kw):
    from paper_2206_04993_gb300 import Solver
    return Solver(kind=S.SGEP_CCA, d_x=dx, d_y=dx, k=k, dtype=S.SGEP_BF16, path=S.SGEP_PATH_TC,
                  debug=1, **kw)


@pytest.mark.parametrize("dx,k,b", [(256, 32, 128), (512, 32, 256), (512, 8, 384), (768, 17, 256)])
def test_tc_single_step_matches_oracle(dx, k, b):
    model = synth.planted_cca(dx, dx, np.linspace(0.9, 0.3, 8), seed=dx + k)
    X, Y = synth.draw_rows(model, b, batch=3)
    V0 = synth.random_unit_columns(2 * dx, k, seed=k)
    S0 = 0.8 * V0 + 0.05 * synth.random_unit_columns(2 * dx, k, seed=k + 1)
    with _tc_solver(dx, k, eta0=0.3, gamma0=0.4, rho=1e-3, max_b=512) as s:
        assert s.path == S.SGEP_PATH_TC
        err = step_errors(s, V0, S0, X, Y, "cca", 0.3, 0.4, 1e-3, dtype="bf16")
    print(err)
    for name, e in err.items():
        assert e <= TC_TOL, (name, e, err)


def test_tc_and_generic_agree_over_steps():
    """Fifty steps of the tensor-core and generic paths on the same BF16 minibatches."""
    from paper_2206_04993_gb300 import Solver
    model = synth.planted_cca(512, 512, np.linspace(0.9, 0.3, 16), seed=5)
    X, Y = synth.draw_rows(model, 256 * 50, batch=1)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda().to(torch.bfloat16)
    Yd = torch.from_numpy(Y.astype(np.float32)).cuda().to(torch.bfloat16)
    V0 = synth.random_unit_columns(1024, 16, seed=2).astype(np.float32)
    out = []
    for path in (S.SGEP_PATH_GENERIC, S.SGEP_PATH_TC):
        with Solver(kind=S.SGEP_CCA, d_x=512, d_y=512, k=16, dtype=S.SGEP_BF16, path=path,
                    eta0=0.2, gamma0=0.5, max_b=256) as s:
            s.set_V(V0)
            s.step_many(Xd, Yd, 256, 50)
            out.append(s.V())
    assert np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0]) < 1e-3


@pytest.mark.slow
def test_tc_full_size_step_matches_oracle():
    """One step at the full activation-like shape (d_x = d_y = 16384, k = 32, b = 4096)."""
    cfg = synth.config_c3()
    X, Y = synth.draw_rows(cfg["model"], 4096, batch=0, dtype=np.float32)
    V0 = synth.random_unit_columns(32768, 32, seed=0)
    S0 = 0.8 * V0 + 0.05 * synth.random_unit_columns(32768, 32, seed=1)
    with _tc_solver(16384, 32, eta0=0.3, gamma0=0.3, rho=1e-6, max_b=4096) as s:
        err = step_errors(s, V0, S0, X, Y, "cca", 0.3, 0.3, 1e-6, dtype="bf16")
    print(err)
    for name, e in err.items():
        assert e <= TC_TOL, (name, e, err)
