"""Pins of the warm-start oracle (oracle/warm.py) against finite differences and invariances."""
import numpy as np

from oracle import warm


def _params(rng, m=16, h=64, k=5):
    return [rng.standard_normal((h, m)) * 0.3, rng.standard_normal(h) * 0.1, rng.standard_normal((h, h)) * 0.15,
            rng.standard_normal(h) * 0.1, rng.standard_normal((k, h)) * 0.2, rng.standard_normal(k) * 0.1]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    params = _params(rng, m=6, h=9, k=3)
    S = [rng.standard_normal((11, 6)), rng.standard_normal((7, 6))]
    V = [rng.standard_normal((11, 3)), rng.standard_normal((7, 3))]
    loss, grads = warm.loss_and_grads(params, S, V)
    h = 1e-6
    for p, g in zip(params, grads):
        flat = p.reshape(-1)
        num = np.zeros_like(flat)
        for j in range(flat.size):
            keep = flat[j]
            flat[j] = keep + h
            lp, _ = warm.loss_and_grads(params, S, V)
            flat[j] = keep - h
            lm, _ = warm.loss_and_grads(params, S, V)
            flat[j] = keep
            num[j] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g.reshape(-1), num, rtol=1e-5, atol=1e-8)


def test_loss_is_sign_and_scale_invariant_and_zero_at_target():
    rng = np.random.default_rng(1)
    V = rng.standard_normal((20, 4))
    assert abs(warm.loss_instance(V, V)) < 1e-14
    assert abs(warm.loss_instance(V * np.array([-2.0, 3.0, -0.5, 1.0]), V)) < 1e-14
    O = rng.standard_normal((20, 4))
    assert 0.0 < warm.loss_instance(O, V) < 4.0


def test_sketch_is_normalised_covariance_times_omega():
    rng = np.random.default_rng(2)
    X, Y = rng.standard_normal((50, 7)), rng.standard_normal((50, 5))
    om = rng.standard_normal((12, 4))
    S = warm.sketch(X, Y, om)
    Z = np.hstack([X, Y])
    C = Z.T @ Z / 50
    R = C @ om
    np.testing.assert_allclose(S, R / np.sqrt(np.mean(R * R, axis=0)), rtol=1e-12)
    np.testing.assert_allclose(np.mean(S * S, axis=0), 1.0, rtol=1e-12)
