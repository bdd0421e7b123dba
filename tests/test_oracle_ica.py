"""Pins of the oracle's ICA pencil (Sec. 1, ICA): the population closed form against a
brute-force expectation over a discrete source law, the streamed operators against the
explicit finite-sample pencil, unbiasedness of the quarter split, and the unmixing
directions as generalized eigenvectors."""
import itertools

import numpy as np

import synth
from oracle import eg, gep


def _discrete_law(law):
    """Support and probabilities of a discrete unit-variance source law."""
    if law == "rademacher":
        return np.array([-1.0, 1.0]), np.array([0.5, 0.5])
    if law == "sparse":
        return np.array([-2.0, 0.0, 2.0]), np.array([0.125, 0.75, 0.125])
    raise ValueError(law)


def test_population_pencil_matches_brute_force_expectation():
    """E[<x,x> x x^T] - tr(B) B - 2 B^2 and E[x x^T] summed over every source outcome of a
    discrete law equal the closed form M diag(kappa_j |m_j|^2) M^T, M M^T."""
    laws = ["rademacher", "sparse", "sparse", "rademacher"]
    model = synth.planted_ica(4, laws, seed=3)
    M = model["M"]
    supports = [_discrete_law(l) for l in laws]
    E4 = np.zeros((4, 4))
    E2 = np.zeros((4, 4))
    for combo in itertools.product(*[range(len(sp[0])) for sp in supports]):
        s = np.array([supports[j][0][c] for j, c in enumerate(combo)])
        p = np.prod([supports[j][1][c] for j, c in enumerate(combo)])
        x = M @ s
        E4 += p * (x @ x) * np.outer(x, x)
        E2 += p * np.outer(x, x)
    A_bf = E4 - np.trace(E2) * E2 - 2.0 * E2 @ E2
    A, B = gep.ica_population_AB(model)
    np.testing.assert_allclose(B, E2, atol=1e-12)
    np.testing.assert_allclose(A, A_bf, atol=1e-11)
    np.testing.assert_allclose(model["kurtosis"], [-2.0, 1.0, 1.0, -2.0])


def test_unsplit_operators_equal_the_finite_sample_pencil(rng):
    model = synth.planted_ica(5, ["laplace", "uniform", "sparse", "rademacher", "gauss"], seed=1)
    X = synth.draw_ica_rows(model, 50, batch=2)
    A, B = gep.form_ica_AB(X)
    Amv, Bmv = eg.ica_ops(X, split=False)
    U = rng.standard_normal((5, 3))
    np.testing.assert_allclose(Amv(U), A @ U, atol=1e-10)
    np.testing.assert_allclose(Bmv(U), B @ U, atol=1e-12)


def test_split_operators_are_unbiased(rng):
    """Alg. 2 needs unbiased A_t and B_t: averaged over many minibatches the quarter-split
    estimates approach the population products within their Monte Carlo error (5 sigma)."""
    model = synth.planted_ica(3, ["sparse", "uniform", "rademacher"], seed=7)
    A, B = gep.ica_population_AB(model)
    U = rng.standard_normal((3, 2))
    nb, b = 6000, 16
    ests_A = np.empty((nb, 3, 2))
    ests_B = np.empty((nb, 3, 2))
    for t in range(nb):
        Amv, Bmv = eg.ica_ops(synth.draw_ica_rows(model, b, batch=100 + t))
        ests_A[t] = Amv(U)
        ests_B[t] = Bmv(U)
    for est, ref in ((ests_A, A @ U), (ests_B, B @ U)):
        se = est.std(axis=0) / np.sqrt(nb)
        assert np.all(np.abs(est.mean(axis=0) - ref) <= 5 * se + 1e-12), (est.mean(axis=0), ref, se)


def test_unmixing_rows_are_the_generalized_eigenvectors():
    """With B = M M^T the pencil's eigenvectors are the rows of M^-1 (the unmixing directions)
    and the eigenvalues kappa_j |m_j|^2; the top ones are those of the positive-kurtosis sources."""
    model = synth.planted_ica(5, ["laplace", "sparse", "uniform", "rademacher", "gauss"], seed=2)
    A, B = gep.ica_population_AB(model)
    M = model["M"]
    lam_cf = model["kurtosis"] * np.sum(M * M, axis=0)
    lam, V = gep.gep_topk(A, B, 2)
    order = np.argsort(-lam_cf)[:2]
    np.testing.assert_allclose(lam, lam_cf[order], rtol=1e-10)
    W = np.linalg.inv(M)[order].T
    W /= np.linalg.norm(W, axis=0)
    np.testing.assert_allclose(np.abs(np.sum(W * V, axis=0)), [1.0, 1.0], atol=1e-10)


def _update_bias_z(split, n_mc=8000, b=16):
    """Largest |mean update direction - population update direction| in standard errors, over
    n_mc minibatches of b rows (fixed V and [Bv])."""
    model = synth.planted_ica(3, ["sparse", "uniform", "rademacher"], seed=7)
    A, B = gep.ica_population_AB(model)
    V = synth.random_unit_columns(3, 2, seed=1)
    S = B @ V + 0.05 * synth.random_unit_columns(3, 2, seed=2)
    _, _, ref = eg.eg_step(V, S, *eg.matrix_ops(A, B), 0.0, 0.0, rho=1e-6, return_parts=True)
    acc = np.zeros_like(V)
    acc2 = np.zeros_like(V)
    for t in range(n_mc):
        X = synth.draw_ica_rows(model, b, batch=100 + t)
        _, _, p = eg.eg_step(V, S, *eg.ica_ops(X, split=split), 0.0, 0.0, rho=1e-6, return_parts=True)
        acc += p["grad"]
        acc2 += p["grad"] ** 2
    mean = acc / n_mc
    se = np.sqrt(np.maximum(acc2 / n_mc - mean ** 2, 0) / n_mc)
    return float(np.max(np.abs(mean - ref["grad"]) / (se + 1e-12)))


def test_split_update_direction_is_unbiased():
    """The update multiplies A_t terms by B_t terms (Alg. 2), so besides each being unbiased
    they must come from independent rows: with the quarter split the expected update direction
    equals the population one within 5 standard errors."""
    assert _update_bias_z(split=True) < 5.0


def test_unsplit_update_direction_is_biased():
    """The check above has the power to see a dependence: with every term on the same rows
    (the finite-sample pencil of a small minibatch) the expected update is far off."""
    assert _update_bias_z(split=False) > 10.0
