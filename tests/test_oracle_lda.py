"""Pins of the LDA reading of the oracle (running class means, between/within-class
operators) against identities that do not go through the oracle's own code."""
import numpy as np

from oracle import eg, gep
import synth


def _between_scatter(X, labels, C):
    """Between-class scatter of a finite set, written from boolean masks."""
    n = X.shape[0]
    mu = X.mean(axis=0)
    A = np.zeros((X.shape[1], X.shape[1]))
    for c in range(C):
        Xc = X[labels == c]
        if len(Xc):
            m = Xc.mean(axis=0) - mu
            A += (len(Xc) / n) * np.outer(m, m)
    return A


def test_streamed_means_give_between_class_scatter():
    model = synth.planted_lda(12, n_classes=5, seed=1)
    C, d = 5, 12
    sums, counts = np.zeros((C, d)), np.zeros(C)
    rows, labs = [], []
    for t in range(7):
        X, lab = synth.draw_lda_rows(model, 64, batch=t)
        sums, counts = eg.lda_stats_update(sums, counts, X, lab)
        rows.append(X)
        labs.append(lab)
    X, lab = np.concatenate(rows), np.concatenate(labs)
    mean, prior = eg.lda_state(sums, counts)
    np.testing.assert_allclose(prior, np.bincount(lab, minlength=C) / len(lab), rtol=1e-15)
    Amv, _ = eg.lda_ops(X[:2], lab[:2], mean, prior)
    A = Amv(np.eye(d))
    np.testing.assert_allclose(A, _between_scatter(X, lab, C), atol=1e-12)


def test_lda_ops_total_variance_identity():
    """With the batch's own class means, A + B is the batch covariance about its mean."""
    model = synth.planted_lda(9, n_classes=4, seed=3)
    X, lab = synth.draw_lda_rows(model, 300, batch=0)
    C = 4
    mean = np.stack([X[lab == c].mean(axis=0) for c in range(C)])
    prior = np.bincount(lab, minlength=C) / len(lab)
    Amv, Bmv = eg.lda_ops(X, lab, mean, prior, split=False)
    I = np.eye(9)
    Xc = X - X.mean(axis=0)
    np.testing.assert_allclose(Amv(I) + Bmv(I), Xc.T @ Xc / len(X), atol=1e-12)


def test_lda_split_uses_the_second_half_for_B():
    model = synth.planted_lda(6, n_classes=3, seed=4)
    X, lab = synth.draw_lda_rows(model, 40, batch=2)
    mean = np.stack([model["means"][c] for c in range(3)])
    prior = np.full(3, 1 / 3)
    _, Bmv = eg.lda_ops(X, lab, mean, prior, split=True)
    Xt = X[20:] - mean[lab[20:]]
    U = np.random.default_rng(0).standard_normal((6, 2))
    np.testing.assert_allclose(Bmv(U), Xt.T @ (Xt @ U) / 20, atol=1e-12)


def test_unseen_class_has_zero_prior_and_mean():
    mean, prior = eg.lda_state(np.ones((3, 2)), np.array([2.0, 0.0, 2.0]))
    np.testing.assert_array_equal(mean[1], 0.0)
    assert prior[1] == 0.0 and abs(prior.sum() - 1.0) < 1e-15


def test_lda_population_isotropic_reduces_to_between_class_eig():
    """B = s^2 I: generalized eigenpairs are those of A with eigenvalues divided by s^2;
    A has rank C - 1, so the C-th eigenvalue is 0."""
    d, C, s = 10, 4, 0.7
    rng = np.random.default_rng(5)
    means = rng.standard_normal((C, d))
    means -= means.mean(axis=0)
    model = {"means": means, "L": s * np.eye(d), "seed": 0}
    A, B = gep.lda_population_AB(model)
    lam, V = gep.gep_topk(A, B, C)
    w, U = np.linalg.eigh(means.T @ means / C)
    np.testing.assert_allclose(lam[:C - 1], w[::-1][:C - 1] / s ** 2, rtol=1e-10)
    assert abs(lam[C - 1]) < 1e-10
    np.testing.assert_allclose(np.abs(np.sum(V[:, :C - 1] * U[:, ::-1][:, :C - 1], axis=0)), 1.0, atol=1e-8)
