"""GPU test of the bounded device-side waits: a wait that nothing completes gives up after its
limit, the kernel returns, and the host reads SGEP_ETIMEOUT; the context stays usable.

The wait is the grid barrier of the fused tensor-core update (no asynchronous copy is in flight
there). SGEP_TEST_STALL=1 at handle creation makes that barrier wait for one arrival more than
the grid sends, with a 20 ms limit, so every block gives up, records the timeout bit of the
device error word and returns. No GPU fault, trap or hang is involved.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2206_04993_gb300 import Solver, sgep as S  # noqa: E402

import synth  # noqa: E402


def _rows(dx, b, seed):
    model = synth.planted_cca(dx, dx, np.linspace(0.9, 0.3, 8), seed=seed)
    X, Y = synth.draw_rows(model, b, batch=1)
    return (torch.from_numpy(X.astype(np.float32)).cuda().to(torch.bfloat16),
            torch.from_numpy(Y.astype(np.float32)).cuda().to(torch.bfloat16))


def _solver():
    # d_x = 256: the two-pass tensor-core products and the fused update kernel
    return Solver(kind=S.SGEP_CCA, d_x=256, d_y=256, k=8, dtype=S.SGEP_BF16, path=S.SGEP_PATH_TC,
                  eta0=0.2, gamma0=0.5, max_b=256)


def test_stalled_barrier_reports_timeout_and_context_stays_usable(monkeypatch):
    X, Y = _rows(256, 256, seed=31)
    monkeypatch.setenv("SGEP_TEST_STALL", "1")
    with _solver() as s:
        assert s.path == S.SGEP_PATH_TC
        s.step(X, Y)
        with pytest.raises(S.SgepError) as err:
            s.sync()
        assert err.value.status == S.SGEP_ETIMEOUT
        # the error is reported once; the flag is cleared
        s.sync()
    monkeypatch.delenv("SGEP_TEST_STALL")
    torch.cuda.synchronize()  # the device still answers
    with _solver() as s:
        V0 = synth.random_unit_columns(512, 8, seed=2).astype(np.float32)
        s.set_V(V0)
        for _ in range(3):
            s.step(X, Y)
        s.sync()
        V = s.V()
    assert np.all(np.isfinite(V))
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0, atol=1e-5)
