"""Pins of the oracle's Alg. 2 with M machines (`eg.eg_step_machines`).

Alg. 2 averages per-machine update directions and auxiliary increments. The pins below tie it
to facts that do not come from the function itself: with one machine it is Alg. 2's step; with
identical shards the average is that of identical copies; the auxiliary step is linear in B_tm,
so with equal-size shards it equals the auxiliary step with B_t estimated on all rows; the
update direction is not linear (it multiplies A_tm and B_tm terms), so two different shards
give the average of two single-shard directions and not the direction of the pooled rows; and
at the exact solution (every machine holding the population A, B) the step is stationary.
"""
import numpy as np

import synth
from oracle import eg, gep


def _state(d, k, seed):
    V = synth.random_unit_columns(d, k, seed=seed)
    S = 0.8 * V + 0.1 * synth.random_unit_columns(d, k, seed=seed + 1)
    return V, S


def _shards(model, b, M, batch):
    X, Y = synth.draw_rows(model, b * M, batch=batch)
    return X, Y, [(X[m * b:(m + 1) * b], Y[m * b:(m + 1) * b]) for m in range(M)]


def test_one_machine_is_alg2_step():
    model = synth.planted_cca(6, 5, [0.9, 0.7, 0.5], seed=1)
    X, Y = synth.draw_rows(model, 64, batch=0)
    V, S = _state(11, 3, 2)
    V1, S1 = eg.eg_step_machines(V, S, [eg.cca_ops(X, Y)], 0.3, 0.4, 1e-3)
    V2, S2 = eg.eg_step(V, S, *eg.cca_ops(X, Y), 0.3, 0.4, 1e-3)
    np.testing.assert_allclose(V1, V2, rtol=0, atol=1e-14)
    np.testing.assert_allclose(S1, S2, rtol=0, atol=1e-14)


def test_identical_shards_equal_one_shard():
    model = synth.planted_cca(7, 4, [0.9, 0.6], seed=3)
    X, Y = synth.draw_rows(model, 40, batch=1)
    V, S = _state(11, 2, 4)
    ops = eg.cca_ops(X, Y)
    V3, S3 = eg.eg_step_machines(V, S, [ops, ops, ops], 0.2, 0.5, 1e-3)
    V1, S1 = eg.eg_step(V, S, *ops, 0.2, 0.5, 1e-3)
    np.testing.assert_allclose(V3, V1, atol=1e-13)
    np.testing.assert_allclose(S3, S1, atol=1e-13)


def test_aux_step_is_linear_and_direction_is_not():
    """Two different equal-size shards: [Bv]' equals the pooled-rows [Bv]' (B_t V is linear in
    the rows), while the direction is the mean of the two shard directions, written out here
    with the explicit block matrices of each shard (not through the oracle's operators)."""
    dx, dy, k, b = 5, 4, 3, 32
    model = synth.planted_cca(dx, dy, [0.9, 0.6, 0.4], seed=5)
    X, Y, shards = _shards(model, b, 2, batch=2)
    V, S = _state(dx + dy, k, 6)
    eta, gamma, rho = 0.25, 0.35, 1e-3
    Vm, Sm = eg.eg_step_machines(V, S, [eg.cca_ops(x, y) for x, y in shards], eta, gamma, rho)
    # auxiliary step: B estimated on the B halves of both shards together
    XB = np.concatenate([x[b // 2:] for x, _ in shards])
    YB = np.concatenate([y[b // 2:] for _, y in shards])
    B = np.zeros((dx + dy, dx + dy))
    B[:dx, :dx] = XB.T @ XB / XB.shape[0]
    B[dx:, dx:] = YB.T @ YB / YB.shape[0]
    np.testing.assert_allclose(Sm, S + gamma * (B @ V - S), atol=1e-12)
    # direction: per shard, the matrix form of Eq. (update) with explicit A_m, B_m
    grads = []
    for x, y in shards:
        xa, ya, xb, yb = x[:b // 2], y[:b // 2], x[b // 2:], y[b // 2:]
        A = np.zeros((dx + dy, dx + dy))
        A[:dx, dx:] = xa.T @ ya / (b // 2)
        A[dx:, :dx] = A[:dx, dx:].T
        Bm = np.zeros_like(A)
        Bm[:dx, :dx] = xb.T @ xb / (b // 2)
        Bm[dx:, dx:] = yb.T @ yb / (b // 2)
        g = np.zeros_like(V)
        for i in range(k):
            vi = V[:, i]
            g[:, i] = (vi @ Bm @ vi) * (A @ vi) - (vi @ A @ vi) * (Bm @ vi)
            for j in range(i):
                sj = max(V[:, j] @ S[:, j], rho)
                g[:, i] -= (vi @ A @ V[:, j] / sj) * ((vi @ Bm @ vi) * S[:, j] - (vi @ S[:, j]) * (Bm @ vi))
        grads.append(g)
    Vp = V + eta * 0.5 * (grads[0] + grads[1])
    np.testing.assert_allclose(Vm, Vp / np.linalg.norm(Vp, axis=0), atol=1e-12)
    # and the pooled rows give a different direction (products of per-shard estimates)
    Vpool, _ = eg.eg_step(V, S, *eg.cca_ops(X, Y), eta, gamma, rho)
    assert np.linalg.norm(Vpool - Vm) > 1e-6


def test_fixed_point_with_population_estimates():
    """Every machine holding the exact A, B: at (V*, [Bv] = B V*) the step leaves V unchanged."""
    rng = np.random.default_rng(7)
    d, k = 6, 3
    Q = rng.standard_normal((d, d))
    B = Q @ Q.T / d + np.eye(d)
    R = rng.standard_normal((d, d))
    A = R + R.T
    lam, Vs = gep.gep_topk(A, B, k)
    Vs = Vs / np.linalg.norm(Vs, axis=0)
    ops = eg.matrix_ops(A, B)
    V1, S1 = eg.eg_step_machines(Vs, B @ Vs, [ops] * 4, 0.1, 0.5, 1e-6)
    np.testing.assert_allclose(np.abs(np.sum(V1 * Vs, axis=0)), 1.0, atol=1e-10)
    np.testing.assert_allclose(S1, B @ Vs, atol=1e-12)
