"""O1: the exact top-k symmetric generalized eigenproblem, in float64.

Test infrastructure only (see the package header).

Route (Prop. "Similar Matrices", App. A): with B = L L^T (Cholesky), the
matrix C = L^-1 A L^-T is symmetric and has the generalized eigenvalues of
(A, B); its orthonormal eigenvectors W map back through V = L^-T W. The
eigenvectors of C are found with the cyclic Jacobi method (Golub & Van Loan,
"Matrix Computations", Sec. 8.5), using the round-robin ordering so that each
round applies n/2 disjoint rotations at once.

Pins (tests/test_oracle_gep.py): the worked 2x2 example of App. B (angle of
about 71 degrees between the generalized eigenvectors, Fig. 1 caption), the
2x2 characteristic polynomial det(A - lambda B) = 0, diagonal A and B,
B = I against LAPACK's symmetric eigensolver, scipy's generalized solver,
B-orthogonality (Lemma "B-orthogonality"), the planted-CCA closed form, and
the paper's pseudo-inverse form of the subspace error (App. A.1).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# Dense building blocks

def cholesky(B: np.ndarray) -> np.ndarray:
    """Lower-triangular L with B = L L^T (column-by-column textbook algorithm)."""
    B = np.asarray(B, dtype=np.float64)
    n = B.shape[0]
    L = np.zeros_like(B)
    for j in range(n):
        s = B[j, j] - L[j, :j] @ L[j, :j]
        if not s > 0.0:
            raise np.linalg.LinAlgError("B is not positive definite")
        L[j, j] = np.sqrt(s)
        L[j + 1:, j] = (B[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def forward_substitute(L: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Solve L Z = M for lower-triangular L (all columns of M at once)."""
    n = L.shape[0]
    Z = np.zeros_like(M, dtype=np.float64)
    for i in range(n):
        Z[i] = (M[i] - L[i, :i] @ Z[:i]) / L[i, i]
    return Z


def back_substitute_transposed(L: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Solve L^T Z = M for lower-triangular L."""
    n = L.shape[0]
    Z = np.zeros_like(M, dtype=np.float64)
    for i in range(n - 1, -1, -1):
        Z[i] = (M[i] - L[i + 1:, i] @ Z[i + 1:]) / L[i, i]
    return Z


def jacobi_eigh(C: np.ndarray, tol: float = 1e-14, max_sweeps: int = 60):
    """Eigen-decomposition of a symmetric matrix by cyclic Jacobi rotations.

    Returns (w, W) with C W = W diag(w), W orthogonal, w in no particular order.
    Each rotation zeroes one off-diagonal pair (p, q): with
    tau = (c_qq - c_pp) / (2 c_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
    c = 1 / sqrt(1 + t^2), s = t c, the update is C <- J^T C J with
    J_pp = J_qq = c, J_pq = s, J_qp = -s. Sweeps stop when the off-diagonal
    Frobenius norm falls below tol times the Frobenius norm of C.
    """
    A = np.array(C, dtype=np.float64, copy=True)
    n = A.shape[0]
    W = np.eye(n)
    if n == 1:
        return A.diagonal().copy(), W
    m = n + (n % 2)
    ring = list(range(m))
    fro = np.linalg.norm(A)
    for _ in range(max_sweeps):
        off = np.linalg.norm(A - np.diag(np.diag(A)))
        if off <= tol * fro or fro == 0.0:
            break
        for _round in range(m - 1):
            pairs = [(ring[i], ring[m - 1 - i]) for i in range(m // 2)]
            pairs = [(min(a, b), max(a, b)) for a, b in pairs if a < n and b < n]
            p = np.array([a for a, _ in pairs])
            q = np.array([b for _, b in pairs])
            apq = A[p, q]
            app = A[p, p]
            aqq = A[q, q]
            nz = apq != 0.0
            t = np.zeros_like(apq)
            tau = np.where(nz, (aqq - app) / np.where(nz, 2.0 * apq, 1.0), 0.0)
            sgn = np.where(tau >= 0.0, 1.0, -1.0)
            t = np.where(nz, sgn / (np.abs(tau) + np.sqrt(1.0 + tau * tau)), 0.0)
            c = 1.0 / np.sqrt(1.0 + t * t)
            s = t * c
            # columns: A <- A J, W <- W J
            Ap, Aq = A[:, p].copy(), A[:, q].copy()
            A[:, p] = c * Ap - s * Aq
            A[:, q] = s * Ap + c * Aq
            Wp, Wq = W[:, p].copy(), W[:, q].copy()
            W[:, p] = c * Wp - s * Wq
            W[:, q] = s * Wp + c * Wq
            # rows: A <- J^T A
            Ap, Aq = A[p, :].copy(), A[q, :].copy()
            A[p, :] = c[:, None] * Ap - s[:, None] * Aq
            A[q, :] = s[:, None] * Ap + c[:, None] * Aq
            ring = [ring[0]] + [ring[-1]] + ring[1:-1]
    return A.diagonal().copy(), W


def gep_topk(A: np.ndarray, B: np.ndarray, k: int):
    """Top-k generalized eigenpairs of (A, B), B symmetric positive definite.

    Returns (lam, V): lam descending, V d x k with unit Euclidean columns
    (the strategy space of Sec. 2 is the unit sphere). Signs are fixed so that
    the largest-magnitude entry of each column is positive.
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    L = cholesky(B)
    Z = forward_substitute(L, A)            # L^-1 A
    C = forward_substitute(L, Z.T)          # L^-1 A^T L^-T = L^-1 A L^-T
    C = 0.5 * (C + C.T)
    w, W = jacobi_eigh(C)
    order = np.argsort(-w)[:k]
    lam = w[order]
    V = back_substitute_transposed(L, W[:, order])
    V /= np.linalg.norm(V, axis=0, keepdims=True)
    idx = np.argmax(np.abs(V), axis=0)
    V *= np.sign(V[idx, np.arange(V.shape[1])])[None, :]
    return lam, V


# ---------------------------------------------------------------------------
# A and B of the problem kinds (Sec. 1), formed explicitly from a finite sample.
# Data are assumed zero-mean; means are 1/n (Sec. 1, "means over a finite
# sample dataset").

def form_cca_AB(X: np.ndarray, Y: np.ndarray):
    """A = [[0, E xy^T], [E yx^T, 0]], B = blockdiag(E xx^T, E yy^T) (Sec. 1, CCA)."""
    n, dx = X.shape
    dy = Y.shape[1]
    d = dx + dy
    A = np.zeros((d, d))
    B = np.zeros((d, d))
    A[:dx, dx:] = X.T @ Y / n
    A[dx:, :dx] = Y.T @ X / n
    B[:dx, :dx] = X.T @ X / n
    B[dx:, dx:] = Y.T @ Y / n
    return A, B


def form_pca_AB(X: np.ndarray):
    """A = X^T X / n, B = I (Sec. 1, PCA)."""
    n, d = X.shape
    return X.T @ X / n, np.eye(d)


def form_pls_AB(X: np.ndarray, Y: np.ndarray):
    """PLS: A as for CCA, B = I (reading of the sentence in Sec. 1 naming PLS)."""
    A, _ = form_cca_AB(X, Y)
    return A, np.eye(A.shape[0])


def form_lda_AB(X: np.ndarray, labels: np.ndarray, n_classes: int):
    """LDA: between-class scatter A and within-class covariance B (reading; Sec. 1 names LDA).

    A = sum_c pi_c (mu_c - mu)(mu_c - mu)^T, B = (1/n) sum_r (x_r - mu_{l_r})(x_r - mu_{l_r})^T.
    """
    n, d = X.shape
    mu = X.mean(axis=0)
    A = np.zeros((d, d))
    Xc = X.astype(np.float64).copy()
    for c in range(n_classes):
        sel = labels == c
        if not np.any(sel):
            continue
        pc = sel.mean()
        mc = X[sel].mean(axis=0)
        A += pc * np.outer(mc - mu, mc - mu)
        Xc[sel] -= mc
    return A, Xc.T @ Xc / n


# ---------------------------------------------------------------------------
# Closed forms for the planted models

def lda_population_AB(model):
    """Population A (between-class, equal priors) and B (shared within-class L L^T) of planted LDA."""
    means = np.asarray(model["means"], dtype=np.float64)
    C = means.shape[0]
    mu = means.mean(axis=0)
    Mc = means - mu[None, :]
    A = Mc.T @ Mc / C
    L = np.asarray(model["L"], dtype=np.float64)
    return A, L @ L.T


def form_ica_AB(X: np.ndarray):
    """ICA pencil of a finite set (Sec. 1, ICA): B = mean x x^T and
    A = mean <x, x> x x^T - tr(B) B - 2 B^2 (excess kurtosis matrix)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    B = X.T @ X / n
    w = np.einsum("rd,rd->r", X, X)
    A = (X * w[:, None]).T @ X / n - np.trace(B) * B - 2.0 * B @ B
    return 0.5 * (A + A.T), B


def ica_population_AB(model):
    """Population ICA pencil of x = M s with independent unit-variance sources of excess
    kurtosis kappa_j: B = M M^T, and the contraction of the fourth cumulant of x over one pair
    of indices gives A = M diag(kappa_j |m_j|^2) M^T, so the generalized eigenvectors are the
    rows of M^-1 with eigenvalues kappa_j |m_j|^2."""
    M = np.asarray(model["M"], dtype=np.float64)
    kap = np.asarray(model["kurtosis"], dtype=np.float64)
    A = (M * (kap * np.sum(M * M, axis=0))[None, :]) @ M.T
    return 0.5 * (A + A.T), M @ M.T


def cca_population_AB(model):
    """Population A and B of a planted CCA model (x = W_x z + noise, y = W_y z + noise)."""
    if hasattr(model, "sigma"):
        Wx, Wy = model.Qx * model.s, model.Qy * model.s
        Cxx = Wx @ Wx.T + model.sigma ** 2 * np.eye(Wx.shape[0])
        Cyy = Wy @ Wy.T + model.sigma ** 2 * np.eye(Wy.shape[0])
    else:
        Wx, Wy = model.Wx, model.Wy
        Cxx = Wx @ Wx.T + np.diag(model.Dx)
        Cyy = Wy @ Wy.T + np.diag(model.Dy)
    dx, dy = Wx.shape[0], Wy.shape[0]
    d = dx + dy
    A = np.zeros((d, d))
    B = np.zeros((d, d))
    A[:dx, dx:] = Wx @ Wy.T
    A[dx:, :dx] = Wy @ Wx.T
    B[:dx, :dx] = Cxx
    B[dx:, dx:] = Cyy
    return A, B


def cca_truth_lowrank(Dx, Dy, Wx, Wy, k: int):
    """Top-k generalized eigenpairs of population CCA with Cxx = diag(Dx) + Wx Wx^T, Cxy = Wx Wy^T.

    With v = [a; b], A v = lambda B v reads Wx Wy^T b = lambda Cxx a and
    Wy Wx^T a = lambda Cyy b. Writing alpha = Wx^T a and beta = Wy^T b gives
    lambda^2 alpha = G_x G_y alpha with G = W^T C^-1 W = H (I + H)^-1 and
    H = W^T D^-1 W (Woodbury). The m x m problem is symmetrised as
    G_x^{1/2} G_y G_x^{1/2} u = lambda^2 u with alpha = G_x^{1/2} u; then
    beta = G_y alpha / lambda, a = D^-1 Wx (I + H_x)^-1 beta / lambda and
    b = D^-1 Wy (I + H_y)^-1 alpha / lambda. Cost O(d m^2).
    Returns (lam descending, V d x k with unit Euclidean columns).
    """
    Dx = np.asarray(Dx, dtype=np.float64)
    Dy = np.asarray(Dy, dtype=np.float64)
    m = Wx.shape[1]
    Im = np.eye(m)
    Hx = Wx.T @ (Wx / Dx[:, None])
    Hy = Wy.T @ (Wy / Dy[:, None])
    Gx = Hx @ np.linalg.inv(Im + Hx)
    Gy = Hy @ np.linalg.inv(Im + Hy)
    Gx = 0.5 * (Gx + Gx.T)
    Gy = 0.5 * (Gy + Gy.T)
    wx, Ux = jacobi_eigh(Gx)
    Gx_half = (Ux * np.sqrt(np.maximum(wx, 0.0))[None, :]) @ Ux.T
    M = Gx_half @ Gy @ Gx_half
    w2, U = jacobi_eigh(0.5 * (M + M.T))
    order = np.argsort(-w2)[:k]
    lam = np.sqrt(np.maximum(w2[order], 0.0))
    alpha = Gx_half @ U[:, order]
    beta = (Gy @ alpha) / lam[None, :]
    a = (Wx / Dx[:, None]) @ np.linalg.solve(Im + Hx, beta) / lam[None, :]
    b = (Wy / Dy[:, None]) @ np.linalg.solve(Im + Hy, alpha) / lam[None, :]
    V = np.vstack([a, b])
    V /= np.linalg.norm(V, axis=0, keepdims=True)
    idx = np.argmax(np.abs(V), axis=0)
    V *= np.sign(V[idx, np.arange(V.shape[1])])[None, :]
    return lam, V


def cca_truth_from_covariances(Cxx, Cyy, Cxy, k: int):
    """Top-k CCA pairs from the covariance blocks through LAPACK (the paper's ground truth is
    scipy's symmetric generalized solver, Sec. 5). With Cxx = Lx Lx^T, Cyy = Ly Ly^T, the
    generalized eigenvalues of the CCA pencil are +-singular values of K = Lx^-1 Cxy Ly^-T and
    the eigenvectors are [Lx^-T u; Ly^-T w] for the singular pairs (u, w) (Prop. "Similar
    Matrices" applied blockwise). Returns (lam descending, V with unit Euclidean columns)."""
    Lx = np.linalg.cholesky(np.asarray(Cxx, dtype=np.float64))
    Ly = np.linalg.cholesky(np.asarray(Cyy, dtype=np.float64))
    import scipy.linalg as sla
    K = sla.solve_triangular(Lx, np.asarray(Cxy, dtype=np.float64), lower=True)
    K = sla.solve_triangular(Ly, K.T, lower=True).T
    U, sv, Wt = np.linalg.svd(K)
    a = sla.solve_triangular(Lx.T, U[:, :k], lower=False)
    b = sla.solve_triangular(Ly.T, Wt[:k].T, lower=False)
    V = np.vstack([a, b])
    V /= np.linalg.norm(V, axis=0, keepdims=True)
    idx = np.argmax(np.abs(V), axis=0)
    V *= np.sign(V[idx, np.arange(V.shape[1])])[None, :]
    return sv[:k], V


def cca_truth_planted(model, k: int):
    """Top-k truth of a PlantedCCA model (orthonormal Q, isotropic noise sigma^2).

    Cxx^-1/2 Cxy Cyy^-1/2 = sum_l q_xl q_yl^T s_l^2 / (s_l^2 + sigma^2), so the
    canonical correlations are s_l^2 / (s_l^2 + sigma^2) and the unit-norm
    generalized eigenvectors are [q_xl; q_yl] / sqrt(2).
    """
    rho = model.s ** 2 / (model.s ** 2 + model.sigma ** 2)
    order = np.argsort(-rho)[:k]
    V = np.vstack([model.Qx[:, order], model.Qy[:, order]]) / np.sqrt(2.0)
    return rho[order], V


def cca_B_apply(model, U: np.ndarray) -> np.ndarray:
    """B U for a planted CCA model without forming B (O(d m k))."""
    if hasattr(model, "sigma"):
        Wx, Wy = model.Qx * model.s, model.Qy * model.s
        dx = Wx.shape[0]
        ux, uy = U[:dx], U[dx:]
        return np.vstack([Wx @ (Wx.T @ ux) + model.sigma ** 2 * ux,
                          Wy @ (Wy.T @ uy) + model.sigma ** 2 * uy])
    dx = model.Wx.shape[0]
    ux, uy = U[:dx], U[dx:]
    return np.vstack([model.Wx @ (model.Wx.T @ ux) + model.Dx[:, None] * ux,
                      model.Wy @ (model.Wy.T @ uy) + model.Dy[:, None] * uy])


# ---------------------------------------------------------------------------
# Evaluation (App. A.1)

def subspace_error(V_true: np.ndarray, V_hat: np.ndarray, B) -> float:
    """Generalized subspace error 1 - tr(U* P) / k (App. A.1).

    U* and P are the orthogonal projectors onto span(B^{1/2} V_true) and
    span(B^{1/2} V_hat). Writing them through Gram matrices removes B^{1/2}:
    tr(U* P) = tr[(Vt^T B Vt)^-1 (Vt^T B Vh) (Vh^T B Vh)^-1 (Vh^T B Vt)].
    `B` is a matrix or a callable returning B U.
    """
    Bop = B if callable(B) else (lambda U: np.asarray(B) @ U)
    BVt = Bop(V_true)
    BVh = Bop(V_hat)
    Gtt = V_true.T @ BVt
    Ghh = V_hat.T @ BVh
    Gth = V_true.T @ BVh
    k = V_true.shape[1]
    tr = np.trace(np.linalg.solve(Gtt, Gth) @ np.linalg.solve(Ghh, Gth.T))
    return float(1.0 - tr / k)


def rayleigh_quotients(V: np.ndarray, A, B) -> np.ndarray:
    """lambda_hat_i = <v_i, A v_i> / <v_i, B v_i> (Sec. 2, below Eq. util_new)."""
    Aop = A if callable(A) else (lambda U: np.asarray(A) @ U)
    Bop = B if callable(B) else (lambda U: np.asarray(B) @ U)
    return np.sum(V * Aop(V), axis=0) / np.sum(V * Bop(V), axis=0)
