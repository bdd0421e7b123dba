"""Pins of the oracle's algorithm variants: Adam on the players (App. H.2.2) and the smooth
denominators of Alg. 3 (App. E.2), against closed forms, finite differences, the clipped
Alg. 2 step and the fixed point of the method."""
import numpy as np
import pytest

from oracle import eg, gep


def _problem(rng, d=10, k=4, b=64):
    X = rng.standard_normal((b, d // 2))
    Y = 0.6 * X @ rng.standard_normal((d // 2, d // 2)) / np.sqrt(d) + rng.standard_normal((b, d // 2))
    V = rng.standard_normal((d, k))
    V /= np.linalg.norm(V, axis=0)
    S = 0.7 * V + 0.1 * rng.standard_normal((d, k))
    return X, Y, V, S


def test_smooth_denominator_closed_forms():
    """Alg. 3: sigmoid(0) = 1/2 gives the geometric mean of rho and nu; the map is increasing
    and tends to rho and nu at -inf and +inf."""
    rho, nu = 1e-4, 25.0
    np.testing.assert_allclose(eg.smooth_denominator(np.zeros(1), rho, nu), [np.sqrt(rho * nu)], rtol=1e-14)
    s = eg.smooth_denominator(np.linspace(-20, 20, 81), rho, nu)
    assert np.all(np.diff(s) > 0)
    ends = eg.smooth_denominator(np.array([-60.0, 60.0]), rho, nu)
    np.testing.assert_allclose(ends, [rho, nu], rtol=1e-12)


def test_smooth_step_equals_clipped_step_at_matching_denominators(rng):
    """With z chosen so that s_j = max(<v_j, [Bv]_j>, rho), Alg. 3 takes the players and the
    auxiliary variables exactly where Alg. 2 takes them."""
    X, Y, V, S = _problem(rng)
    Amv, Bmv = eg.cca_ops(X, Y)
    rho, nu = 1e-3, 50.0
    target = np.maximum(np.einsum("dk,dk->k", V, S), rho)
    sig = (np.log(target) - np.log(rho)) / (np.log(nu) - np.log(rho))
    z = np.log(sig / (1.0 - sig))
    V1, S1 = eg.eg_step(V, S, Amv, Bmv, 0.2, 0.4, rho)
    V2, S2, st = eg.eg_step_variant(V, S, Amv, Bmv, 0.2, 0.4, rho, smooth={"z": z, "nu": nu})
    np.testing.assert_allclose(V2, V1, atol=1e-12)
    np.testing.assert_allclose(S2, S1, atol=1e-12)


def test_smooth_z_step_descends_the_squared_mismatch(rng):
    """The z step of Alg. 3 is gamma times minus the derivative of (s(z) - <v, [Bv]>)^2 / 2
    (central differences), and z stays put when s(z) already equals <v, [Bv]>."""
    X, Y, V, S = _problem(rng)
    Amv, Bmv = eg.cca_ops(X, Y)
    rho, nu, gamma = 1e-3, 20.0, 0.3
    z = rng.standard_normal(V.shape[1])
    c = np.einsum("dk,dk->k", V, S)
    _, _, st = eg.eg_step_variant(V, S, Amv, Bmv, 0.1, gamma, rho, smooth={"z": z, "nu": nu})
    h = 1e-6
    for i in range(z.size):
        def f(zi):
            return 0.5 * (eg.smooth_denominator(np.array([zi]), rho, nu)[0] - c[i]) ** 2
        deriv = (f(z[i] + h) - f(z[i] - h)) / (2 * h)
        np.testing.assert_allclose((st["smooth"]["z"][i] - z[i]) / gamma, -deriv, rtol=1e-6, atol=1e-10)
    # at s(z) = <v, [Bv]> (positive entries only) the z step vanishes
    cpos = np.clip(c, 2 * rho, nu / 2)
    S2 = S * (cpos / c)[None, :]
    sig = (np.log(cpos) - np.log(rho)) / (np.log(nu) - np.log(rho))
    z0 = np.log(sig / (1.0 - sig))
    _, _, st0 = eg.eg_step_variant(V, S2, Amv, Bmv, 0.1, gamma, rho, smooth={"z": z0, "nu": nu})
    np.testing.assert_allclose(st0["smooth"]["z"], z0, atol=1e-12)


def test_no_variant_is_alg2(rng):
    X, Y, V, S = _problem(rng)
    Amv, Bmv = eg.cca_ops(X, Y)
    V1, S1 = eg.eg_step(V, S, Amv, Bmv, 0.2, 0.4, 1e-4)
    V2, S2, st = eg.eg_step_variant(V, S, Amv, Bmv, 0.2, 0.4, 1e-4)
    np.testing.assert_allclose(V2, V1, atol=1e-14)
    np.testing.assert_allclose(S2, S1, atol=1e-14)
    assert st == {}


def _adam(d, k, b1=0.9, b2=0.999, eps=1e-8):
    return {"m": np.zeros((d, k)), "s": np.zeros((d, k)), "t": 0, "b1": b1, "b2": b2, "eps": eps}


def test_adam_first_step_is_normalised_gradient(rng):
    """With zero moments the bias-corrected first moment is g and the second g^2, so the first
    Adam step moves every coordinate by eta g / (|g| + eps)."""
    X, Y, V, S = _problem(rng)
    Amv, Bmv = eg.cca_ops(X, Y)
    eta, eps = 0.05, 1e-3
    _, _, parts = eg.eg_step(V, S, Amv, Bmv, eta, 0.4, 1e-4, return_parts=True)
    g = parts["grad"]
    Vp = V + eta * g / (np.abs(g) + eps)
    V2, S2, st = eg.eg_step_variant(V, S, Amv, Bmv, eta, 0.4, 1e-4, adam=_adam(*V.shape, eps=eps))
    np.testing.assert_allclose(V2, Vp / np.linalg.norm(Vp, axis=0), atol=1e-13)
    assert st["adam"]["t"] == 1


def test_adam_without_momentum_repeats_the_normalised_step(rng):
    """b1 = b2 = 0: every step (not only the first) moves by eta g / (|g| + eps)."""
    X, Y, V, S = _problem(rng)
    Amv, Bmv = eg.cca_ops(X, Y)
    eta, eps = 0.05, 1e-2
    ad = _adam(*V.shape, b1=0.0, b2=0.0, eps=eps)
    V1, S1, st = eg.eg_step_variant(V, S, Amv, Bmv, eta, 0.4, 1e-4, adam=ad)
    _, _, parts = eg.eg_step(V1, S1, Amv, Bmv, eta, 0.4, 1e-4, return_parts=True)
    g = parts["grad"]
    Vp = V1 + eta * g / (np.abs(g) + eps)
    V2, _, _ = eg.eg_step_variant(V1, S1, Amv, Bmv, eta, 0.4, 1e-4, adam=st["adam"])
    np.testing.assert_allclose(V2, Vp / np.linalg.norm(Vp, axis=0), atol=1e-13)


def test_adam_trajectory_equals_a_library_adam(rng):
    """Six chained Adam steps equal torch.optim.Adam (the textbook recursion, run on the CPU in
    FP64) given the same update directions (negated: torch descends) and the same retraction:
    momentum decay, bias correction over t and the epsilon's place all have to match."""
    torch = pytest.importorskip("torch")
    X, Y, V, S = _problem(rng)
    Amv, Bmv = eg.cca_ops(X, Y)
    eta, gamma, rho, b1, b2, eps = 0.05, 0.4, 1e-4, 0.8, 0.95, 1e-3
    p = torch.nn.Parameter(torch.tensor(V, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=eta, betas=(b1, b2), eps=eps)
    ad = _adam(*V.shape, b1=b1, b2=b2, eps=eps)
    Vo, So = V.copy(), S.copy()
    for _ in range(6):
        _, _, parts = eg.eg_step(Vo, So, Amv, Bmv, eta, gamma, rho, return_parts=True)
        p.grad = torch.tensor(-parts["grad"], dtype=torch.float64)
        opt.step()
        with torch.no_grad():
            p /= p.norm(dim=0, keepdim=True)
        Vo, So, st = eg.eg_step_variant(Vo, So, Amv, Bmv, eta, gamma, rho, adam=ad)
        ad = st["adam"]
        np.testing.assert_allclose(Vo, p.detach().numpy(), atol=1e-12)
    assert ad["t"] == 6


def test_adam_keeps_the_solution(rng):
    """App. C fixed point: with exact A, B and [Bv] = B v the update direction is zero (up to
    rounding, which Adam scales by at most 1/eps), so Adam moves neither the players nor its
    moments."""
    d, k = 10, 3
    M = rng.standard_normal((d, d))
    A = M + M.T + 2.0 * np.diag(np.linspace(4, 0, d))
    N = rng.standard_normal((d, d))
    B = N @ N.T / d + 0.5 * np.eye(d)
    lam, Vs = gep.gep_topk(A, B, k)
    Amv, Bmv = eg.matrix_ops(A, B)
    V1, S1, st = eg.eg_step_variant(Vs, B @ Vs, Amv, Bmv, 0.3, 0.5, 1e-8, adam=_adam(d, k, eps=1e-4))
    np.testing.assert_allclose(V1, Vs, atol=1e-8)
    assert np.abs(st["adam"]["m"]).max() < 1e-10


def test_adam_is_invariant_to_scaling_A(rng):
    """The update direction is linear in A (rewards and penalties each carry one factor of
    A_t), and Adam with eps = 0 divides that scale out: three steps with A and with 7 A agree."""
    X, Y, V, S = _problem(rng)
    Amv, Bmv = eg.cca_ops(X, Y)

    def run(scale):
        A7 = (lambda U: scale * Amv(U))
        Vc, Sc, ad = V, S, _adam(*V.shape, eps=0.0)
        for _ in range(3):
            Vc, Sc, st = eg.eg_step_variant(Vc, Sc, A7, Bmv, 0.05, 0.4, 1e-4, adam=ad)
            ad = st["adam"]
        return Vc

    np.testing.assert_allclose(run(7.0), run(1.0), atol=1e-12)
