"""Pins of the Rayleigh-Ritz correction in the oracle."""
import numpy as np

from oracle import eg, gep


def _pencil(rng, d):
    M = rng.standard_normal((d, d))
    A = M + M.T
    N = rng.standard_normal((d, d))
    B = N @ N.T + d * np.eye(d)
    return A, B


def test_exact_subspace_is_rotated_onto_the_eigenvectors():
    """If span(V) is the top-k eigenspace, Rayleigh-Ritz returns the eigenvectors themselves."""
    rng = np.random.default_rng(0)
    d, k = 20, 4
    A, B = _pencil(rng, d)
    w, U = __import__("scipy.linalg", fromlist=["eigh"]).eigh(A, B)
    Vstar = U[:, ::-1][:, :k]
    V = Vstar @ rng.standard_normal((k, k))
    V /= np.linalg.norm(V, axis=0)
    Amv, Bmv = eg.matrix_ops(A, B)
    Vn, Sn, lam = eg.rayleigh_ritz(V, B @ V, Amv, Bmv)
    np.testing.assert_allclose(lam, w[::-1][:k], rtol=1e-10)
    Vs = Vstar / np.linalg.norm(Vstar, axis=0)
    np.testing.assert_allclose(np.abs(np.sum(Vn * Vs, axis=0)), 1.0, atol=1e-10)
    np.testing.assert_allclose(Sn, B @ Vn, atol=1e-10)  # S = B V is carried exactly


def test_ritz_vectors_are_B_orthogonal_and_span_is_kept():
    rng = np.random.default_rng(1)
    d, k = 15, 5
    A, B = _pencil(rng, d)
    V = rng.standard_normal((d, k))
    V /= np.linalg.norm(V, axis=0)
    Vn, _, lam = eg.rayleigh_ritz(V, V.copy(), *eg.matrix_ops(A, B))
    G = Vn.T @ B @ Vn
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-10 * np.abs(np.diag(G)).max()
    assert gep.subspace_error(V, Vn, B) < 1e-12
    assert np.all(np.diff(lam) <= 0)
    np.testing.assert_allclose(gep.rayleigh_quotients(Vn, A, B), lam, rtol=1e-10)
    np.testing.assert_allclose(np.linalg.norm(Vn, axis=0), 1.0, rtol=1e-14)
