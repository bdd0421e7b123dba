"""Helpers shared by the GPU tests: run one library step and the oracle step on the same
inputs and compute the relative errors the parity tests bound."""
from __future__ import annotations

import numpy as np

from oracle import eg

# Per-step parity bar for the FP32 path (relative to the magnitude of the terms).
STEP_TOL = 1e-5
# The per-column checks (keys ending in "_col" and "_elem") bound what a whole-matrix
# Frobenius ratio dilutes: an error confined to one player column or to a few rows (a ragged
# tail tile). One column's rounding error relative to its own norm, and the largest element
# error relative to the column's largest entry, may exceed the whole-matrix ratio by a small
# factor (a column of small norm; the maximum of d errors against the maximum of d values),
# so those keys are held to COL_FACTOR times the step bar.
COL_FACTOR = 4.0


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even to bfloat16, returned as float32 (the values the GPU reads)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def to_device(a: np.ndarray, dtype: str):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return t.to(torch.bfloat16) if dtype == "bf16" else t


def oracle_ops(kind: str, X, Y, split: bool, eps_B: float):
    X = np.asarray(X, dtype=np.float64)
    if kind == "pca":
        return eg.pca_ops(X, eps_B)
    Y = np.asarray(Y, dtype=np.float64)
    if kind == "pls":
        return eg.pls_ops(X, Y, eps_B)
    return eg.cca_ops(X, Y, split=split, eps_B=eps_B)


def rel(a, b) -> float:
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0))


def col_errors(a, b):
    """(max over columns of |a_i - b_i| / |b_i|, max over columns of max_c |a_ci - b_ci| /
    max_c |b_ci|) for d x k matrices whose columns are players."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    diff = np.abs(a - b)
    nb = np.linalg.norm(b, axis=0)
    mb = np.max(np.abs(b), axis=0)
    col = np.linalg.norm(a - b, axis=0) / np.where(nb > 0, nb, 1.0)
    elem = np.max(diff, axis=0) / np.where(mb > 0, mb, 1.0)
    return float(np.max(col)), float(np.max(elem))


def assert_within(err: dict, tol: float):
    """Every whole-matrix ratio within tol, every per-column ratio within COL_FACTOR tol."""
    for name, e in err.items():
        lim = tol * (COL_FACTOR if name.endswith(("_col", "_elem")) else 1.0)
        assert e <= lim, (name, e, lim, err)


def step_errors(solver, V0, S0, X, Y, kind, eta, gamma, rho, split=True, eps_B=0.0, dtype="f32"):
    """Run one library step from (V0, S0) on (X, Y) and one oracle step on the same values.
    Returns a dict of relative errors for A_t V, B_t V, grad, V', S'."""
    import torch
    Xv = bf16_round(X) if dtype == "bf16" else np.asarray(X, np.float32)
    Yv = None if Y is None else (bf16_round(Y) if dtype == "bf16" else np.asarray(Y, np.float32))
    V0 = np.asarray(V0, np.float32)
    S0 = np.asarray(S0, np.float32)
    solver.set_V(V0, S0)
    Xd = to_device(Xv, dtype)
    Yd = None if Yv is None else to_device(Yv, dtype)
    solver.step(Xd, Yd)
    AVg, BVg = solver.products()
    torch.cuda.synchronize()
    Vg = solver.V()
    Sg = solver.S()
    Amv, Bmv = oracle_ops(kind, Xv, Yv, split, eps_B)
    V1, S1, parts = eg.eg_step(V0.astype(np.float64), S0.astype(np.float64), Amv, Bmv,
                               eta, gamma, rho, return_parts=True)
    AV, BV, grad = parts["AV"], parts["BV"], parts["grad"]
    out = {"AV": rel(AVg, AV), "V": rel(Vg, V1), "S": rel(Sg, S1)}
    if kind == "cca":
        out["BV"] = rel(BVg, BV - eps_B * V0.astype(np.float64))
        out["BV_col"], out["BV_elem"] = col_errors(BVg, BV - eps_B * V0.astype(np.float64))
    out["AV_col"], out["AV_elem"] = col_errors(AVg, AV)
    out["V_col"], out["V_elem"] = col_errors(Vg, V1)
    out["S_col"], out["S_elem"] = col_errors(Sg, S1)
    if solver.cfg.debug:
        gg, a, G, b = solver.update_terms()
        a_ref = V0.astype(np.float64).T @ AV
        bvec = np.sum(V0 * BV, axis=0)
        reward = AV * bvec - BV * np.diag(a_ref)
        scale = (np.linalg.norm(AV * bvec) + np.linalg.norm(BV * np.diag(a_ref))
                 + np.linalg.norm(reward - grad))
        out["grad"] = float(np.linalg.norm(gg - grad) / scale)
        out["a"] = rel(a, a_ref)
        out["G"] = rel(G, V0.astype(np.float64).T @ S0)
        out["b"] = rel(b, bvec)
    return out
