"""Pins of the O1 oracle (exact top-k generalized eigenproblem) against facts fixed by the
paper and by mathematics, independent of the oracle's own code."""
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import eg, gep
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_worked_example():
    A, B, angle = [], [], None
    with open(os.path.join(GOLDEN, "worked_example_2x2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tag, *vals = line.split()
            if tag == "A":
                A.append([float(v) for v in vals])
            elif tag == "B":
                B.append([float(v) for v in vals])
            elif tag == "angle_deg":
                angle = (float(vals[0]), float(vals[1]))
    return np.array(A), np.array(B), angle


def _quadratic_gep_2x2(A, B):
    # det(A - l B) = 0  <=>  det(B) l^2 - (a11 b22 + a22 b11 - 2 a12 b12) l + det(A) = 0
    a2 = B[0, 0] * B[1, 1] - B[0, 1] ** 2
    a1 = -(A[0, 0] * B[1, 1] + A[1, 1] * B[0, 0] - 2 * A[0, 1] * B[0, 1])
    a0 = A[0, 0] * A[1, 1] - A[0, 1] ** 2
    disc = np.sqrt(a1 * a1 - 4 * a2 * a0)
    return np.array([(-a1 + disc) / (2 * a2), (-a1 - disc) / (2 * a2)])


def test_worked_example_angle_and_utilities():
    """App. B example / Fig. 1: eigenvectors ~71 degrees apart; u_2 is 0 at v_1 and lambda_2 at v_2."""
    A, B, (angle, tol) = _load_worked_example()
    lam, V = gep.gep_topk(A, B, 2)
    ang = np.degrees(np.arccos(abs(V[:, 0] @ V[:, 1])))
    assert abs(ang - angle) <= tol
    np.testing.assert_allclose(lam, _quadratic_gep_2x2(A, B), rtol=1e-12)
    aligned_with_v1 = np.stack([V[:, 0], V[:, 0]], axis=1)
    assert abs(eg.utility(aligned_with_v1, 1, A, B)) < 1e-12
    assert abs(eg.utility(V, 1, A, B) - lam[1]) < 1e-12 * lam[0]


def test_characteristic_polynomial_2x2(rng):
    for _ in range(20):
        M = rng.standard_normal((2, 2))
        A = M + M.T
        N = rng.standard_normal((2, 2))
        B = N @ N.T + 0.1 * np.eye(2)
        lam, V = gep.gep_topk(A, B, 2)
        np.testing.assert_allclose(lam, _quadratic_gep_2x2(A, B), rtol=1e-10, atol=1e-12)
        for i in range(2):
            r = A @ V[:, i] - lam[i] * B @ V[:, i]
            assert np.linalg.norm(r) < 1e-10 * (np.linalg.norm(A) + abs(lam[i]) * np.linalg.norm(B))


def test_diagonal_pencil(rng):
    """Diagonal A and B: lambda_i = a_ii / b_ii and the eigenvectors are unit coordinate vectors."""
    d, k = 9, 5
    a = rng.uniform(-1, 3, d)
    bdiag = rng.uniform(0.2, 2, d)
    lam, V = gep.gep_topk(np.diag(a), np.diag(bdiag), k)
    ratio = a / bdiag
    order = np.argsort(-ratio)[:k]
    np.testing.assert_allclose(lam, ratio[order], rtol=1e-12)
    np.testing.assert_allclose(np.abs(V), np.eye(d)[:, order], atol=1e-12)


def test_identity_B_matches_lapack(rng):
    d, k = 30, 6
    M = rng.standard_normal((d, d))
    A = M + M.T
    lam, V = gep.gep_topk(A, np.eye(d), k)
    w, U = np.linalg.eigh(A)
    np.testing.assert_allclose(lam, w[::-1][:k], rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(np.abs(V.T @ U[:, ::-1][:, :k]), np.eye(k), atol=1e-9)


def test_general_pencil_matches_scipy(rng):
    d, k = 40, 7
    M = rng.standard_normal((d, d))
    A = M + M.T
    N = rng.standard_normal((d, d))
    B = N @ N.T + d * np.eye(d)
    lam, V = gep.gep_topk(A, B, k)
    w, U = sl.eigh(A, B)
    np.testing.assert_allclose(lam, w[::-1][:k], rtol=1e-10)
    assert gep.subspace_error(U[:, ::-1][:, :k], V, B) < 1e-12


def test_b_orthogonality_and_rayleigh(rng):
    """Lemma "B-orthogonality": V^T B V is diagonal and V^T A V = Lambda V^T B V."""
    d, k = 25, 8
    M = rng.standard_normal((d, d))
    A = M + M.T
    N = rng.standard_normal((d, d))
    B = N @ N.T + 0.5 * np.eye(d)
    lam, V = gep.gep_topk(A, B, k)
    G = V.T @ B @ V
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-10 * np.abs(np.diag(G)).max()
    np.testing.assert_allclose(V.T @ A @ V, np.diag(lam) @ G, atol=1e-9 * np.abs(lam).max())
    np.testing.assert_allclose(gep.rayleigh_quotients(V, A, B), lam, rtol=1e-10)


def test_cholesky_and_triangular_solves(rng):
    d = 20
    N = rng.standard_normal((d, d))
    B = N @ N.T + np.eye(d)
    L = gep.cholesky(B)
    np.testing.assert_allclose(L @ L.T, B, atol=1e-11)
    np.testing.assert_allclose(L, np.linalg.cholesky(B), atol=1e-11)
    M = rng.standard_normal((d, 3))
    np.testing.assert_allclose(L @ gep.forward_substitute(L, M), M, atol=1e-10)
    np.testing.assert_allclose(L.T @ gep.back_substitute_transposed(L, M), M, atol=1e-10)
    with pytest.raises(np.linalg.LinAlgError):
        gep.cholesky(-np.eye(3))


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33, 64])
def test_jacobi_matches_lapack(rng, n):
    M = rng.standard_normal((n, n))
    C = M + M.T
    w, W = gep.jacobi_eigh(C)
    np.testing.assert_allclose(np.sort(w), np.linalg.eigvalsh(C), atol=1e-11 * max(1, n))
    assert np.abs(W.T @ W - np.eye(n)).max() < 1e-12 * max(1, n)
    assert np.abs(C @ W - W * w).max() < 1e-11 * max(1, n)


def test_jacobi_repeated_eigenvalues():
    w, W = gep.jacobi_eigh(3.0 * np.eye(5))
    np.testing.assert_allclose(w, 3.0)
    Q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((6, 6)))
    C = Q @ np.diag([2, 2, 2, -1, -1, 5.0]) @ Q.T
    w, W = gep.jacobi_eigh(C)
    np.testing.assert_allclose(np.sort(w), [-1, -1, 2, 2, 2, 5], atol=1e-12)


def test_planted_cca_closed_form():
    """Planted CCA: canonical correlations s^2/(s^2+sigma^2) and vectors [q_x; q_y]/sqrt(2)."""
    rhos = np.array([0.9, 0.75, 0.6, 0.45, 0.3, 0.2])
    model = synth.planted_cca(24, 20, rhos, sigma=0.5, seed=3)
    A, B = gep.cca_population_AB(model)
    lam, V = gep.gep_topk(A, B, 4)
    lam_cf, V_cf = gep.cca_truth_planted(model, 4)
    np.testing.assert_allclose(lam, lam_cf, rtol=1e-10)
    np.testing.assert_allclose(lam, rhos[:4], rtol=1e-10)
    np.testing.assert_allclose(np.abs(np.sum(V * V_cf, axis=0)), 1.0, atol=1e-10)


def test_lowrank_cca_closed_form():
    """The Woodbury reduction used for the 16384+16384 workload equals the dense solve."""
    model = synth.planted_lowrank_cca(40, 36, m=6, alpha=1.0, seed=5)
    A, B = gep.cca_population_AB(model)
    lam, V = gep.gep_topk(A, B, 4)
    lam_lr, V_lr = gep.cca_truth_lowrank(model.Dx, model.Dy, model.Wx, model.Wy, 4)
    np.testing.assert_allclose(lam_lr, lam, rtol=1e-9)
    np.testing.assert_allclose(np.abs(np.sum(V * V_lr, axis=0)), 1.0, atol=1e-9)
    Bop = lambda U: gep.cca_B_apply(model, U)  # noqa: E731
    np.testing.assert_allclose(Bop(V), B @ V, atol=1e-12)


def test_subspace_error_matches_pseudoinverse_form(rng):
    """App. A.1: 1 - tr(U* P)/k with U* = W W^+, P = W^ W^+^, W = B^{1/2} V."""
    d, k = 15, 4
    N = rng.standard_normal((d, d))
    B = N @ N.T + np.eye(d)
    Bh = np.real(sl.sqrtm(B))
    for _ in range(5):
        Vt = rng.standard_normal((d, k))
        Vh = rng.standard_normal((d, k))
        W = Bh @ Vt
        Wh = Bh @ Vh
        ref = 1 - np.trace((W @ np.linalg.pinv(W)) @ (Wh @ np.linalg.pinv(Wh))) / k
        assert abs(gep.subspace_error(Vt, Vh, B) - ref) < 1e-10
    Vt = rng.standard_normal((d, k))
    R = rng.standard_normal((k, k))
    assert abs(gep.subspace_error(Vt, Vt @ R, B)) < 1e-10            # same span -> 0
    # a B-orthogonal complement -> 1
    L = np.linalg.cholesky(B)
    Q, _ = np.linalg.qr(rng.standard_normal((d, 2 * k)))
    Vt2 = np.linalg.solve(L.T, Q[:, :k])
    Vh2 = np.linalg.solve(L.T, Q[:, k:])
    assert abs(gep.subspace_error(Vt2, Vh2, B) - 1.0) < 1e-10


def test_lda_forms(rng):
    model = synth.planted_lda(6, n_classes=3, seed=2)
    X, labels = synth.draw_lda_rows(model, 500, batch=0)
    A, B = gep.form_lda_AB(X, labels, 3)
    # total covariance = between + within (law of total variance, finite-sample form)
    Xc = X - X.mean(axis=0)
    np.testing.assert_allclose(A + B, Xc.T @ Xc / X.shape[0], atol=1e-12)
    assert np.linalg.matrix_rank(A, tol=1e-10) <= 2


def test_lapack_cca_route_matches_jacobi_oracle(rng):
    """The LAPACK route used for ground truth at d = 1024 equals Cholesky + Jacobi."""
    model = synth.planted_cca(20, 16, [0.9, 0.7, 0.5, 0.3], sigma=0.5, seed=8)
    X, Y = synth.draw_rows(model, 400, batch=2)
    A, B = gep.form_cca_AB(X, Y)
    lam, V = gep.gep_topk(A, B, 4)
    n = X.shape[0]
    lam2, V2 = gep.cca_truth_from_covariances(X.T @ X / n, Y.T @ Y / n, X.T @ Y / n, 4)
    np.testing.assert_allclose(lam2, lam, rtol=1e-10)
    np.testing.assert_allclose(np.abs(np.sum(V * V2, axis=0)), 1.0, atol=1e-9)
