"""Pins of the O2 oracle (the gamma-EigenGame iteration, Alg. 1 and Alg. 2) against facts the
paper proves and against textbook special cases, independent of the oracle's own code."""
import numpy as np
import pytest

from oracle import eg, gep
import synth


def _random_pencil(rng, d):
    M = rng.standard_normal((d, d))
    A = M + M.T + 2.0 * np.diag(np.linspace(4, 0, d))
    N = rng.standard_normal((d, d))
    B = N @ N.T / d + 0.5 * np.eye(d)
    return A, B


def test_update_vanishes_at_solution(rng):
    """App. C: with exact A, B the unique fixed point is the top-k solution with [Bv] = B v."""
    d, k = 12, 5
    A, B = _random_pencil(rng, d)
    lam, Vs = gep.gep_topk(A, B, k)
    Amv, Bmv = eg.matrix_ops(A, B)
    V1, S1, parts = eg.eg_step(Vs, B @ Vs, Amv, Bmv, eta=0.3, gamma=0.5, rho=1e-8, return_parts=True)
    scale = np.abs(lam).max() * np.abs(np.diag(Vs.T @ B @ Vs)).max()
    assert np.abs(parts["grad"]).max() < 1e-12 * scale
    np.testing.assert_allclose(V1, Vs, atol=1e-12)
    np.testing.assert_allclose(S1, B @ Vs, atol=1e-12)


def _numeric_grad(f, x, h=1e-6):
    g = np.zeros_like(x)
    for c in range(x.size):
        e = np.zeros_like(x)
        e[c] = h
        g[c] = (f(x + e) - f(x - e)) / (2 * h)
    return g


def test_update_is_scaled_utility_gradient_with_exact_parents(rng):
    """Lemma "Gradient" (App. B) + relation (i) of Sec. 3: with exact parents and exact [Bv],
    grad_i = <v_i, B v_i>^2 / 2 * d u_i / d v_i (finite differences of Eq. util_new)."""
    d, k = 8, 4
    A, B = _random_pencil(rng, d)
    _, Vs = gep.gep_topk(A, B, k)
    Amv, Bmv = eg.matrix_ops(A, B)
    for i in range(1, k):
        V = Vs.copy()
        vi = rng.standard_normal(d)
        V[:, i] = vi / np.linalg.norm(vi)
        V[:, i + 1:] = rng.standard_normal((d, k - i - 1))
        _, _, parts = eg.eg_step(V, B @ V, Amv, Bmv, eta=0.0, gamma=0.0, rho=1e-12, return_parts=True)

        def u(x):
            W = V.copy()
            W[:, i] = x
            return eg.utility(W, i, A, B)

        g = _numeric_grad(u, V[:, i].copy())
        vBv = V[:, i] @ B @ V[:, i]
        np.testing.assert_allclose(parts["grad"][:, i], 0.5 * vBv ** 2 * g, rtol=1e-6, atol=1e-7)


def test_identity_B_reduces_to_mu_eigengame(rng):
    """Prop. "Equivalence to EigenGame Unloaded": with B = I and [Bv] = v,
    grad_i = (I - v_i v_i^T)[A v_i - sum_{j<i} (v_i^T A v_j) v_j]."""
    d, k = 10, 5
    M = rng.standard_normal((d, d))
    A = M + M.T
    V = rng.standard_normal((d, k))
    V /= np.linalg.norm(V, axis=0)
    Amv, Bmv = eg.matrix_ops(A, np.eye(d))
    _, _, parts = eg.eg_step(V, V.copy(), Amv, Bmv, eta=0.0, gamma=0.0, rho=1e-12, return_parts=True)
    for i in range(k):
        vi = V[:, i]
        r = A @ vi - sum((vi @ A @ V[:, j]) * V[:, j] for j in range(i))
        expect = r - vi * (vi @ r)
        np.testing.assert_allclose(parts["grad"][:, i], expect, atol=1e-12)


def test_retraction_and_auxiliary_special_cases(rng):
    """eta = 0 keeps V; gamma = 1 sets [Bv] to B_t v (the running average restarts);
    repeated identical batches pull [Bv] geometrically toward B_t v; columns stay unit norm."""
    X, Y = synth.draw_rows(synth.planted_cca(7, 5, [0.8, 0.5], seed=1), 40, batch=0)
    Amv, Bmv = eg.cca_ops(X, Y)
    V = synth.random_unit_columns(12, 3, seed=4)
    S = rng.standard_normal((12, 3))
    V1, S1 = eg.eg_step(V, S, Amv, Bmv, eta=0.0, gamma=1.0, rho=1e-6)
    np.testing.assert_allclose(V1, V, atol=1e-15)
    np.testing.assert_allclose(S1, Bmv(V), atol=1e-14)
    S_t = S.copy()
    g = 0.3
    for _ in range(6):
        _, S_t = eg.eg_step(V, S_t, Amv, Bmv, eta=0.0, gamma=g, rho=1e-6)
    np.testing.assert_allclose(S_t - Bmv(V), (1 - g) ** 6 * (S - Bmv(V)), atol=1e-13)
    V2, _ = eg.eg_step(V, S, Amv, Bmv, eta=0.7, gamma=0.2, rho=1e-6)
    np.testing.assert_allclose(np.linalg.norm(V2, axis=0), 1.0, atol=1e-14)


def test_clipping_floor_scales_penalty(rng):
    """Alg. 2 clips <v_j, [Bv]_j> below at rho: when clipped, the penalty is proportional to 1/rho."""
    d, k = 9, 3
    A, B = _random_pencil(rng, d)
    Amv, Bmv = eg.matrix_ops(A, B)
    V = synth.random_unit_columns(d, k, seed=7)
    S = -V.copy()                      # <v_j, [Bv]_j> = -1 < rho
    _, _, p1 = eg.eg_step(V, S, Amv, Bmv, 0.0, 0.0, rho=0.5, return_parts=True)
    _, _, p2 = eg.eg_step(V, S, Amv, Bmv, 0.0, 0.0, rho=1.0, return_parts=True)
    AV, BV = A @ V, B @ V
    reward = np.sum(V * BV, 0) * AV - np.sum(V * AV, 0) * BV
    pen1 = reward - p1["grad"]
    pen2 = reward - p2["grad"]
    # finite and present: without the floor the denominators would be square roots of -1
    assert np.all(np.isfinite(pen1)) and np.all(np.isfinite(pen2))
    assert np.abs(pen1[:, 1:]).max() > 1e-3 * np.abs(reward).max()
    np.testing.assert_allclose(pen1[:, 0], 0.0, atol=1e-13)   # player 1 has no parents
    np.testing.assert_allclose(pen1[:, 1:], 2.0 * pen2[:, 1:], rtol=1e-10, atol=1e-12)


def test_streamed_operators_match_block_matrices(rng):
    """Sec. 1 block forms: CCA A = [[0, XY], [YX, 0]], B = blockdiag(XX, YY); PCA/PLS B = I."""
    b, dx, dy, k = 37, 6, 4, 3
    X = rng.standard_normal((b, dx))
    Y = rng.standard_normal((b, dy))
    U = rng.standard_normal((dx + dy, k))
    nA = b // 2
    Amv, Bmv = eg.cca_ops(X, Y, split=True)
    A_A, _ = gep.form_cca_AB(X[:nA], Y[:nA])
    _, B_B = gep.form_cca_AB(X[nA:], Y[nA:])
    np.testing.assert_allclose(Amv(U), A_A @ U, atol=1e-13)
    np.testing.assert_allclose(Bmv(U), B_B @ U, atol=1e-13)
    Amv, Bmv = eg.cca_ops(X, Y, split=False, eps_B=0.25)
    A_all, B_all = gep.form_cca_AB(X, Y)
    np.testing.assert_allclose(Amv(U), A_all @ U, atol=1e-13)
    np.testing.assert_allclose(Bmv(U), (B_all + 0.25 * np.eye(dx + dy)) @ U, atol=1e-13)
    Amv, Bmv = eg.pca_ops(X)
    np.testing.assert_allclose(Amv(U[:dx]), gep.form_pca_AB(X)[0] @ U[:dx], atol=1e-13)
    np.testing.assert_allclose(Bmv(U[:dx]), U[:dx], atol=0)
    Amv, Bmv = eg.pls_ops(X, Y)
    np.testing.assert_allclose(Amv(U), gep.form_pls_AB(X, Y)[0] @ U, atol=1e-13)


@pytest.mark.slow
def test_split_minibatch_update_is_unbiased():
    """Sec. 3: with independent batches for A_t and B_t the expected update equals the update
    with population A and B (fixed V and [Bv]). Monte Carlo over many minibatches."""
    model = synth.planted_cca(5, 4, [0.9, 0.6, 0.3], sigma=0.5, seed=11)
    A, B = gep.cca_population_AB(model)
    V = synth.random_unit_columns(9, 3, seed=1)
    S = B @ V + 0.05 * synth.random_unit_columns(9, 3, seed=2)
    _, _, ref = eg.eg_step(V, S, *eg.matrix_ops(A, B), 0.0, 0.0, rho=1e-6, return_parts=True)
    n_mc, b = 6000, 8
    acc = np.zeros_like(V)
    acc2 = np.zeros_like(V)
    for t in range(n_mc):
        X, Y = synth.draw_rows(model, b, batch=t)
        _, _, p = eg.eg_step(V, S, *eg.cca_ops(X, Y, split=True), 0.0, 0.0, rho=1e-6, return_parts=True)
        acc += p["grad"]
        acc2 += p["grad"] ** 2
    mean = acc / n_mc
    se = np.sqrt(np.maximum(acc2 / n_mc - mean ** 2, 0) / n_mc)
    z = np.abs(mean - ref["grad"]) / (se + 1e-12)
    assert np.max(z) < 5.0, np.max(z)


def _pencil_with_spectrum(rng, lam):
    """A = L Q diag(lam) Q^T L^T with B = L L^T, so the generalized eigenvalues are lam."""
    d = len(lam)
    N = rng.standard_normal((d, d))
    B = N @ N.T / d + 0.5 * np.eye(d)
    L = np.linalg.cholesky(B)
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    return L @ Q @ np.diag(lam) @ Q.T @ L.T, B


def test_alg1_converges_to_o1():
    """Thm "Deterministic / Full-batch Global Convergence" with eta_t proportional to 1/t."""
    d, k = 8, 3
    A, B = _pencil_with_spectrum(np.random.default_rng(7), [10, 7, 4, 2, 1, 0.5, -1, -2])
    lam, Vs = gep.gep_topk(A, B, k)
    V = synth.random_unit_columns(d, k, seed=3)
    scale = np.linalg.norm(A, 2) * np.linalg.norm(B, 2)
    for t in range(1, 6001):
        V = eg.alg1_step(V, A, B, eta=0.3 / scale * 1000.0 / (t + 1000.0))
    assert gep.subspace_error(Vs, V, B) < 1e-8
    np.testing.assert_allclose(gep.rayleigh_quotients(V, A, B), lam, rtol=1e-5)


def test_alg2_full_batch_converges_to_o1():
    d, k = 10, 4
    A, B = _pencil_with_spectrum(np.random.default_rng(8), [12, 9, 6, 4, 2, 1, 0.5, -1, -2, -3])
    lam, Vs = gep.gep_topk(A, B, k)
    V = synth.random_unit_columns(d, k, seed=9)
    S = V.copy()
    Amv, Bmv = eg.matrix_ops(A, B)
    scale = np.linalg.norm(A, 2) * np.linalg.norm(B, 2)
    for _ in range(4000):
        V, S = eg.eg_step(V, S, Amv, Bmv, eta=0.3 / scale, gamma=0.5, rho=1e-6)
    assert gep.subspace_error(Vs, V, B) < 1e-10
    np.testing.assert_allclose(np.abs(np.sum(V * Vs, axis=0)), 1.0, atol=1e-6)


def test_schedule_endpoints():
    """App. H.2.2: linear warm-up to eta0 at t_c, then 1/(t + Delta) decay reaching eta_T at T."""
    eta0, t_c, T, eta_T = 1e-2, 100, 10_000, 1e-4
    assert eg.schedule_eta(50, eta0, 2, t_c, T, eta_T) == pytest.approx(eta0 * 0.5)
    assert eg.schedule_eta(t_c, eta0, 2, t_c, T, eta_T) == pytest.approx(eta0)
    assert eg.schedule_eta(T, eta0, 2, t_c, T, eta_T) == pytest.approx(eta_T)
    assert eg.schedule_eta(50, eta0, 1, t_c, T, eta_T) == pytest.approx(eta0)
    a, b_, c = (eg.schedule_eta(t, eta0, 1, t_c, T, eta_T) for t in (200, 400, 800))
    # harmonic: 1/eta is affine in t
    assert (1 / c - 1 / b_) == pytest.approx(2 * (1 / b_ - 1 / a), rel=1e-9)
    assert eg.schedule_eta(12345, 0.3, 0) == 0.3


@pytest.mark.slow
def test_stochastic_cca_small_config_reaches_low_error():
    """Alg. 2 on the 4-player CCA workload (finite 10k rows, b = 256): subspace error to the
    finite-sample truth, and the largest eigenvalue error, fall below 1e-3 within 2000 steps."""
    cfg = synth.config_c1()
    X, Y = cfg["X"], cfg["Y"]
    A, B = gep.form_cca_AB(X, Y)
    lam, Vs = gep.gep_topk(A, B, cfg["k"])
    V = synth.random_unit_columns(64, cfg["k"], seed=0)
    S = V.copy()
    for t in range(1, cfg["steps"] + 1):
        idx = synth.finite_dataset_indices(X.shape[0], cfg["b"], t)
        eta = eg.schedule_eta(t, cfg["eta0"], cfg["schedule"], cfg["t_c"], cfg["T"], cfg["eta_T"])
        V, S = eg.eg_step(V, S, *eg.cca_ops(X[idx], Y[idx]), eta, cfg["gamma0"], cfg["rho"])
    err = gep.subspace_error(Vs, V, B)
    assert err < 1e-3, err
    lam_hat = np.array([V[:, j] @ A @ V[:, j] / (V[:, j] @ B @ V[:, j]) for j in range(cfg["k"])])
    assert np.max(np.abs(lam_hat - lam)) < 1e-3, (lam_hat, lam)


def test_running_mean_centring_streams_the_exact_mean_and_removes_offsets():
    """App. H.2.2's learned means: streaming every row of a finite set gives that set's mean,
    and once a constant offset is absorbed by the running mean, centred rows (and so A_t, B_t)
    do not depend on it."""
    model = synth.planted_cca(6, 5, [0.9, 0.6], seed=2)
    rows = [synth.draw_rows(model, 32, batch=b) for b in range(5)]
    X = np.concatenate([r[0] for r in rows])
    sx, n, mx = np.zeros(6), 0.0, None
    for Xb, _ in rows:
        sx, n, mx = eg.running_mean_update(sx, n, Xb)
    np.testing.assert_allclose(mx, X.mean(axis=0), atol=1e-14)
    off = np.linspace(-3.0, 5.0, 6)
    s0, s1, n0, n1 = np.zeros(6), np.zeros(6), 0.0, 0.0
    U = np.random.default_rng(0).standard_normal((11, 3))
    for Xb, Yb in rows:
        s0, n0, m0 = eg.running_mean_update(s0, n0, Xb)
        s1, n1, m1 = eg.running_mean_update(s1, n1, Xb + off)
        A0, B0 = eg.cca_ops(Xb - m0, Yb)
        A1, B1 = eg.cca_ops(Xb + off - m1, Yb)
        np.testing.assert_allclose(A1(U), A0(U), atol=1e-12)
        np.testing.assert_allclose(B1(U), B0(U), atol=1e-12)
