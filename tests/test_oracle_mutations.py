"""Planted mistakes in the oracle's Alg. 2 step must each fail at least one of the independent
pins of test_oracle_eg.py (fixed point at the solution, the utility-gradient relation, the B = I
reduction, the retraction and auxiliary special cases, the clipping floor, full-batch
convergence). A copy of the step with switches (bit-identical to eg.eg_step when no switch is
on) stands in for eg.eg_step while the pins run. Everything here runs on the CPU."""
import numpy as np
import pytest

import test_oracle_eg as pins
from oracle import eg

MISTAKES = [
    "no_penalty",          # the parents' penalty dropped
    "penalty_sign",        # rewards + penalty
    "self_parent",         # j <= i: a player penalised by itself
    "no_sqrt",             # y_j = v_j / <v_j, [Bv]_j> instead of / sqrt(.)
    "no_clip",             # <v_j, [Bv]_j> not floored at rho
    "By_from_v",           # B y_j formed from v_j instead of [Bv]_j
    "vAy_uses_B",          # v_i^T B_t y_j in place of v_i^T A_t y_j
    "reward_uses_A",       # reward's second term with A_t v_i in place of B_t v_i
    "no_retraction",       # v' not renormalised
    "aux_uses_A",          # [Bv] pulled toward A_t v
    "aux_sign",            # [Bv] <- [Bv] + gamma ([Bv] - B_t v)
]


def _step(mistake=None):
    """Alg. 2 (M = 1) with at most one planted mistake."""

    def step(V, S, Amv, Bmv, eta, gamma, rho, return_parts=False):
        V = np.asarray(V, dtype=np.float64)
        S = np.asarray(S, dtype=np.float64)
        d, k = V.shape
        AV = Amv(V)
        BV = Bmv(V)
        grad = np.zeros_like(V)
        for i in range(k):
            vi, Avi, Bvi = V[:, i], AV[:, i], BV[:, i]
            vBv = vi @ Bvi
            vAv = vi @ Avi
            rewards = vBv * Avi - vAv * (Avi if mistake == "reward_uses_A" else Bvi)
            penalties = np.zeros(d)
            for j in range(i + 1 if mistake == "self_parent" else i):
                s = V[:, j] @ S[:, j] if mistake == "no_clip" else max(V[:, j] @ S[:, j], rho)
                denom = s if mistake == "no_sqrt" else np.sqrt(s)
                Byj = (V[:, j] if mistake == "By_from_v" else S[:, j]) / denom
                vAy = vi @ (BV if mistake == "vAy_uses_B" else AV)[:, j] / denom
                penalties += vAy * (vBv * Byj - (vi @ Byj) * Bvi)
            if mistake == "no_penalty":
                penalties[:] = 0.0
            grad[:, i] = rewards + penalties if mistake == "penalty_sign" else rewards - penalties
        Vp = V + eta * grad
        V_next = Vp if mistake == "no_retraction" else Vp / np.linalg.norm(Vp, axis=0, keepdims=True)
        if mistake == "aux_uses_A":
            S_next = S + gamma * (AV - S)
        elif mistake == "aux_sign":
            S_next = S + gamma * (S - BV)
        else:
            S_next = S + gamma * (BV - S)
        if return_parts:
            return V_next, S_next, {"AV": AV, "BV": BV, "grad": grad}
        return V_next, S_next

    return step


PINS = [
    lambda: pins.test_update_vanishes_at_solution(np.random.default_rng(1)),
    lambda: pins.test_update_is_scaled_utility_gradient_with_exact_parents(np.random.default_rng(2)),
    lambda: pins.test_identity_B_reduces_to_mu_eigengame(np.random.default_rng(3)),
    lambda: pins.test_retraction_and_auxiliary_special_cases(np.random.default_rng(4)),
    lambda: pins.test_clipping_floor_scales_penalty(np.random.default_rng(5)),
    pins.test_alg2_full_batch_converges_to_o1,
]


def test_switchable_copy_is_the_oracle_step(rng):
    """With no mistake planted the copy returns exactly what eg.eg_step returns."""
    A, B = pins._random_pencil(rng, 9)
    Amv, Bmv = eg.matrix_ops(A, B)
    V = rng.standard_normal((9, 4))
    S = rng.standard_normal((9, 4))
    for rho in (1e-6, 2.0):  # unclipped and clipped parents
        ref = eg.eg_step(V, S, Amv, Bmv, 0.3, 0.4, rho, return_parts=True)
        got = _step()(V, S, Amv, Bmv, 0.3, 0.4, rho, return_parts=True)
        for x, y in zip(ref[:2], got[:2]):
            assert np.array_equal(x, y)
        for key in ("AV", "BV", "grad"):
            assert np.array_equal(ref[2][key], got[2][key])


def test_pins_pass_with_the_unmutated_copy(monkeypatch):
    monkeypatch.setattr(eg, "eg_step", _step())
    for pin in PINS:
        pin()


@pytest.mark.parametrize("mistake", MISTAKES)
def test_every_planted_mistake_fails_a_pin(mistake, monkeypatch):
    monkeypatch.setattr(eg, "eg_step", _step(mistake))
    failed = []
    with np.errstate(all="ignore"):  # some mistakes produce NaN (the square root of a negative)
        for n, pin in enumerate(PINS):
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError, np.linalg.LinAlgError):
                failed.append(n)
    assert failed, f"no pin caught {mistake}"
