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
from gpu_util import assert_within, step_errors  # noqa: E402

# The tensor-core path multiplies BF16 minibatch values by BF16 (hi, lo) pairs of V and of
# the row projections; a pair carries about 16 significant bits, so each product term has a
# relative error near 2^-17 before FP32 accumulation. The step parity bar for this path is
# therefore 5e-5 (relative, same metric as the FP32 path's 1e-5).
TC_TOL = 5e-5


def _tc_solver(dx, k, dtype=None, **kw):
    from paper_2206_04993_gb300 import Solver
    return Solver(kind=S.SGEP_CCA, d_x=dx, d_y=dx, k=k, dtype=S.SGEP_BF16 if dtype is None else dtype,
                  path=S.SGEP_PATH_TC, debug=1, **kw)


# FP32 rows on the tensor cores: each row value is split into a BF16 pair as well (hi + lo keeps
# about 16 significant bits, |x - hi - lo| <= 2^-16 |x|), and the products add
# X_hi [V_hi | V_lo] + X_lo V_hi. A product term now carries two pair errors near 2^-17 each
# (the row's and V's, or the row's and P's) where a BF16 row carries one, so the products, the
# k x k terms and the update direction get twice the BF16 bar. The update itself, V' and [Bv]'
# (whose change is eta times the direction), keeps the FP32 path's 1e-5.
TC_F32_TOL = 2 * TC_TOL
F32_STEP_TOL = 1e-5


def _assert_f32_step(err):
    upd = {key: v for key, v in err.items() if key[0] in "VS"}
    rest = {key: v for key, v in err.items() if key[0] not in "VS"}
    assert_within(upd, F32_STEP_TOL)
    assert_within(rest, TC_F32_TOL)


@pytest.mark.parametrize("dx,k,b", [(256, 32, 128), (512, 8, 384), (768, 17, 256), (1024, 32, 512)])
def test_tc_f32_rows_single_step_matches_oracle(dx, k, b):
    model = synth.planted_cca(dx, dx, np.linspace(0.9, 0.3, 8), seed=dx + k + 1)
    X, Y = synth.draw_rows(model, b, batch=4)
    V0 = synth.random_unit_columns(2 * dx, k, seed=k + 2)
    S0 = 0.8 * V0 + 0.05 * synth.random_unit_columns(2 * dx, k, seed=k + 3)
    with _tc_solver(dx, k, dtype=S.SGEP_F32, eta0=0.3, gamma0=0.4, rho=1e-3, max_b=512) as s:
        assert s.path == S.SGEP_PATH_TC
        err = step_errors(s, V0, S0, X, Y, "cca", 0.3, 0.4, 1e-3, dtype="f32")
    print(err)
    _assert_f32_step(err)


def test_tc_f32_rows_and_generic_agree_over_steps():
    """Fifty steps of FP32 rows on the tensor cores and on the generic SIMT path."""
    from paper_2206_04993_gb300 import Solver
    model = synth.planted_cca(512, 512, np.linspace(0.9, 0.3, 16), seed=6)
    X, Y = synth.draw_rows(model, 256 * 50, batch=2)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    Yd = torch.from_numpy(Y.astype(np.float32)).cuda()
    V0 = synth.random_unit_columns(1024, 16, seed=3).astype(np.float32)
    out = []
    for path in (S.SGEP_PATH_GENERIC, S.SGEP_PATH_TC):
        with Solver(kind=S.SGEP_CCA, d_x=512, d_y=512, k=16, dtype=S.SGEP_F32, path=path,
                    eta0=0.2, gamma0=0.5, max_b=256) as s:
            s.set_V(V0)
            s.step_many(Xd, Yd, 256, 50)
            out.append(s.V())
    assert np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0]) < 1e-3


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
    assert_within(err, TC_TOL)


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
        # a chained step at this size is one launch: products, row-side terms and update
        Xd = torch.from_numpy(np.asarray(X, np.float32)).cuda().to(torch.bfloat16)
        Yd = torch.from_numpy(np.asarray(Y, np.float32)).cuda().to(torch.bfloat16)
        l0 = s.launches
        s.step(Xd, Yd)
        s.sync()
        assert s.launches - l0 == 1
    print(err)
    assert_within(err, TC_TOL)


@pytest.mark.slow
def test_tc_f32_rows_full_size_step_matches_oracle():
    """FP32 rows at the full activation-like shape (d_x = d_y = 16384, k = 32, b = 4096)."""
    cfg = synth.config_c3()
    X, Y = synth.draw_rows(cfg["model"], 4096, batch=1, dtype=np.float32)
    V0 = synth.random_unit_columns(32768, 32, seed=2)
    S0 = 0.8 * V0 + 0.05 * synth.random_unit_columns(32768, 32, seed=3)
    with _tc_solver(16384, 32, dtype=S.SGEP_F32, eta0=0.3, gamma0=0.3, rho=1e-6, max_b=4096) as s:
        assert s.path == S.SGEP_PATH_TC
        err = step_errors(s, V0, S0, X, Y, "cca", 0.3, 0.3, 1e-6, dtype="f32")
    print(err)
    _assert_f32_step(err)


# Shapes the streamed steps take (d_x a multiple of 512, b of 256): one and several 256-row
# chunks, more row tiles than builder CTAs (d_x = 512, b = 1024), odd k.
@pytest.mark.parametrize("dx,k,b", [(512, 32, 256), (512, 32, 512), (1024, 17, 768), (512, 4, 1024),
                                    (2048, 32, 1024), (1536, 8, 512)])
def test_tc_stream_single_step_matches_oracle(dx, k, b):
    """One step of the streamed path: products, row-side terms and update in one launch."""
    model = synth.planted_cca(dx, dx, np.linspace(0.9, 0.3, 8), seed=dx + k + 1)
    X, Y = synth.draw_rows(model, b, batch=4)
    V0 = synth.random_unit_columns(2 * dx, k, seed=k + 7)
    S0 = 0.8 * V0 + 0.05 * synth.random_unit_columns(2 * dx, k, seed=k + 8)
    with _tc_solver(dx, k, eta0=0.3, gamma0=0.4, rho=1e-3, max_b=b) as s:
        assert s.path == S.SGEP_PATH_TC
        err = step_errors(s, V0, S0, X, Y, "cca", 0.3, 0.4, 1e-3, dtype="bf16")
        # a chained step of the streamed path is one launch
        Xd = torch.from_numpy(X.astype(np.float32)).cuda().to(torch.bfloat16)
        Yd = torch.from_numpy(Y.astype(np.float32)).cuda().to(torch.bfloat16)
        l0 = s.launches
        s.step(Xd, Yd)
        s.sync()
        assert s.launches - l0 == 1
    print(err)
    assert_within(err, TC_TOL)


def _oracle_chain(X, Y, V0, S0, b, n, eta, gamma, rho):
    """n chained oracle steps of Alg. 2 on consecutive b-row minibatches of the BF16 values."""
    from gpu_util import bf16_round
    from oracle import eg
    Xv, Yv = bf16_round(X).astype(np.float64), bf16_round(Y).astype(np.float64)
    V, Sv = V0.astype(np.float64), S0.astype(np.float64)
    parts = None
    for t in range(n):
        V, Sv, parts = eg.eg_step(V, Sv, *eg.cca_ops(Xv[t * b:(t + 1) * b], Yv[t * b:(t + 1) * b]), eta, gamma,
                                  rho, return_parts=True)
    return V, Sv, parts


# Several steps per launch: the retraction of every step but the last is deferred into the
# next step (the next projections are divided by the norms); the chain must equal the
# oracle's chain of normalised steps. Rounding differences grow over the chain by about one
# step's bar per step, so n steps are held to n times the one-step bar.
@pytest.mark.parametrize("dx,k,b,n", [(512, 32, 256, 4), (1024, 17, 512, 3), (512, 8, 768, 5)])
def test_tc_stream_multi_step_launch_matches_oracle(dx, k, b, n):
    model = synth.planted_cca(dx, dx, np.linspace(0.9, 0.3, 8), seed=dx + 3 * k)
    X, Y = synth.draw_rows(model, b * n, batch=6)
    V0 = synth.random_unit_columns(2 * dx, k, seed=k + 11)
    S0 = 0.8 * V0 + 0.05 * synth.random_unit_columns(2 * dx, k, seed=k + 12)
    Vr, Sr, parts = _oracle_chain(X, Y, V0, S0, b, n, 0.3, 0.4, 1e-3)
    with _tc_solver(dx, k, eta0=0.3, gamma0=0.4, rho=1e-3, max_b=b) as s:
        s.set_V(V0.astype(np.float32), S0.astype(np.float32))
        Xd = torch.from_numpy(X.astype(np.float32)).cuda().to(torch.bfloat16)
        Yd = torch.from_numpy(Y.astype(np.float32)).cuda().to(torch.bfloat16)
        l0 = s.launches
        s.step_many(Xd, Yd, b, n)
        s.sync()
        launches = s.launches - l0
        Vg, Sg = s.V(), s.S()
        AVg, BVg = s.products()
        gg, a, G, bb = s.update_terms()
    from gpu_util import col_errors, rel
    err = {"V": rel(Vg, Vr), "S": rel(Sg, Sr), "AV": rel(AVg, parts["AV"]), "BV": rel(BVg, parts["BV"]),
           "grad": rel(gg, parts["grad"])}
    err["V_col"], err["V_elem"] = col_errors(Vg, Vr)
    err["S_col"], err["S_elem"] = col_errors(Sg, Sr)
    print(launches, err)
    assert launches <= 2  # the chain's first step prepares the operand, then one launch
    assert np.allclose(np.linalg.norm(Vg, axis=0), 1.0, atol=1e-5)  # the last step normalises
    assert_within(err, n * TC_TOL)



@pytest.mark.slow
def test_tc_stream_full_size_64_step_launch_matches_oracle():
    """The benchmarked launch: 64 steps of the activation-like shape (d_x = d_y = 16384, k = 32,
    b = 4096, BF16 rows) in one streamed launch, built as the benchmark builds it (no debug
    copies), against 64 oracle steps on the same BF16 values. Four drawn minibatches are taken
    in turn (drawing 64 distinct ones on the host takes minutes); the launch reads each step's
    rows from its own place in device memory either way. Only V and [Bv] are compared, so the
    chain is held to n times the update's one-step bar (1e-5, the bar V' and [Bv]' keep on the
    tensor-core path), not the products' 5e-5."""
    from paper_2206_04993_gb300 import Solver
    from gpu_util import bf16_round, col_errors, rel
    from oracle import eg
    cfg = synth.config_c3()
    b, k, dx, n, m = 4096, 32, 16384, 64, 4
    eta, gamma, rho = 0.3, 0.3, 1e-6
    ops, dev_rows = [], []
    for j in range(m):
        X, Y = synth.draw_rows(cfg["model"], b, batch=20 + j, dtype=np.float32)
        X, Y = bf16_round(X), bf16_round(Y)
        ops.append(eg.cca_ops(X, Y))
        dev_rows.append((torch.from_numpy(X).cuda().to(torch.bfloat16), torch.from_numpy(Y).cuda().to(torch.bfloat16)))
    Xd = torch.empty((n * b, dx), dtype=torch.bfloat16, device="cuda")
    Yd = torch.empty((n * b, dx), dtype=torch.bfloat16, device="cuda")
    for t in range(n):
        Xd[t * b:(t + 1) * b].copy_(dev_rows[t % m][0])
        Yd[t * b:(t + 1) * b].copy_(dev_rows[t % m][1])
    del dev_rows
    V0 = synth.random_unit_columns(2 * dx, k, seed=6).astype(np.float32)
    S0 = (0.8 * V0 + 0.05 * synth.random_unit_columns(2 * dx, k, seed=7)).astype(np.float32)
    Vr, Sr = V0.astype(np.float64), S0.astype(np.float64)
    for t in range(n):
        Vr, Sr = eg.eg_step(Vr, Sr, *ops[t % m], eta, gamma, rho)
    with Solver(kind=S.SGEP_CCA, d_x=dx, d_y=dx, k=k, dtype=S.SGEP_BF16, path=S.SGEP_PATH_TC, eta0=eta,
                gamma0=gamma, rho=rho, max_b=b) as s:
        s.set_V(V0, S0)
        l0 = s.launches
        s.step_many(Xd, Yd, b, n)
        s.sync()
        launches = s.launches - l0
        Vg, Sg = s.V(), s.S()
    err = {"V": rel(Vg, Vr), "S": rel(Sg, Sr)}
    err["V_col"], err["V_elem"] = col_errors(Vg, Vr)
    err["S_col"], err["S_elem"] = col_errors(Sg, Sr)
    print(launches, err)
    assert launches <= 2  # the operand of the first step, then the 64 steps in one launch
    assert np.allclose(np.linalg.norm(Vg, axis=0), 1.0, atol=1e-5)
    assert_within(err, n * F32_STEP_TOL)

def test_tc_stream_steps_beyond_one_launch_match_single_steps():
    """A chain longer than one launch holds (64 steps) equals the same steps taken one call at
    a time (the same arithmetic; only deferred versus immediate retraction rounds differently)."""
    from paper_2206_04993_gb300 import Solver
    dx, k, b, n = 512, 16, 256, 70
    model = synth.planted_cca(dx, dx, np.linspace(0.9, 0.3, 8), seed=21)
    X, Y = synth.draw_rows(model, b * n, batch=7)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda().to(torch.bfloat16)
    Yd = torch.from_numpy(Y.astype(np.float32)).cuda().to(torch.bfloat16)
    V0 = synth.random_unit_columns(2 * dx, k, seed=5).astype(np.float32)
    out = []
    for many in (True, False):
        with Solver(kind=S.SGEP_CCA, d_x=dx, d_y=dx, k=k, dtype=S.SGEP_BF16, path=S.SGEP_PATH_TC, eta0=0.2,
                    gamma0=0.5, max_b=b) as s:
            s.set_V(V0)
            l0 = s.launches
            if many:
                s.step_many(Xd, Yd, b, n)
            else:
                for t in range(n):
                    s.step(Xd[t * b:(t + 1) * b], Yd[t * b:(t + 1) * b])
            s.sync()
            out.append((s.V(), s.S(), s.launches - l0, s.t))
    (Vm, Sm, lm, tm), (V1, S1, l1, t1) = out
    assert tm == t1 == n
    assert lm == 3 and l1 == n + 1, (lm, l1)  # prepare + two launches / prepare + one per step
    assert np.linalg.norm(Vm - V1) / np.linalg.norm(V1) < 1e-4
    assert np.linalg.norm(Sm - S1) / np.linalg.norm(S1) < 1e-4


def test_tc_stream_matches_two_pass_over_steps(monkeypatch):
    """Twenty steps of the streamed products and of the two-pass products on the same
    BF16 minibatches (only the order of the FP32 sums differs)."""
    from paper_2206_04993_gb300 import Solver
    model = synth.planted_cca(1024, 1024, np.linspace(0.9, 0.3, 16), seed=9)
    X, Y = synth.draw_rows(model, 512 * 20, batch=2)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda().to(torch.bfloat16)
    Yd = torch.from_numpy(Y.astype(np.float32)).cuda().to(torch.bfloat16)
    V0 = synth.random_unit_columns(2048, 32, seed=3).astype(np.float32)
    out, launches = [], []
    for env in ("0", "1"):
        monkeypatch.setenv("SGEP_TC_STREAM", env)
        with Solver(kind=S.SGEP_CCA, d_x=1024, d_y=1024, k=32, dtype=S.SGEP_BF16, path=S.SGEP_PATH_TC,
                    eta0=0.2, gamma0=0.5, max_b=512) as s:
            s.set_V(V0)
            l0 = s.launches
            s.step_many(Xd, Yd, 512, 20)
            s.sync()
            launches.append(s.launches - l0)
            out.append(s.V())
    assert launches[1] < launches[0], launches
    assert np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0]) < 1e-4


def test_tc_stream_products_not_kept_without_debug():
    """Without debug the streamed step keeps no A_t V / B_t V; readback says so."""
    from paper_2206_04993_gb300 import Solver
    model = synth.planted_cca(512, 512, np.linspace(0.9, 0.3, 8), seed=4)
    X, Y = synth.draw_rows(model, 256, batch=1)
    with Solver(kind=S.SGEP_CCA, d_x=512, d_y=512, k=8, dtype=S.SGEP_BF16, path=S.SGEP_PATH_TC,
                max_b=256) as s:
        s.step(torch.from_numpy(X.astype(np.float32)).cuda().to(torch.bfloat16),
               torch.from_numpy(Y.astype(np.float32)).cuda().to(torch.bfloat16))
        s.sync()
        with pytest.raises(S.SgepError):
            s.products()
