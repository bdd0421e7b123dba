"""O2: the gamma-EigenGame iteration, written the way the paper states it.

Test infrastructure only (see the package header).

* `eg_step` is one iteration of the stochastic algorithm (Alg. 2) with M = 1
  machine: for every player i it forms y_j and [By]_j of its parents with the
  clipped denominator max(<v_j, [Bv]_j>, rho), the reward and penalty terms of
  Eq. (update) with the minibatch estimates A_t and B_t, the player step
  v_i + eta_t grad_i followed by the retraction to the unit sphere, and the
  auxiliary step [Bv]_i + gamma_t (B_t v_i - [Bv]_i). All players read the
  state of step t (the parfor of Alg. 2), so V and [Bv] are updated together.
* `eg_step_variant` adds the two variants of the paper: Adam on the players with the
  warm-up / harmonic schedule (App. H.2.2) and the smooth denominators of Alg. 3
  (App. E.2, extra scalars z_i).
* `eg_step_machines` is Alg. 2 with M > 1 machines: per-machine update directions and
  auxiliary increments from each machine's own minibatch estimates, averaged.
* `alg1_step` is the deterministic variant (Alg. 1) with exact A and B.
* `utility` is Eq. util_new; `schedule_eta` is the warm-up plus harmonic decay
  of App. H.2.2.
* `ica_ops` is the ICA pencil of Sec. 1 with the quarter reading of independent batches.
* The operators `*_ops` build the minibatch mat-vecs U -> A_t U and U -> B_t U
  from data rows without forming A_t or B_t (Sec. 1: A and B are expectations
  of outer products, applied through matrix-vector products). "Independent
  data batches" for A_t and B_t (Alg. 2) are read as: the first floor(b/2)
  rows estimate A, the other rows estimate B. With B = I (PCA, PLS) no split
  is needed and A uses every row.

Pins (tests/test_oracle_eg.py): the update vanishes at the exact solution with
[Bv] = B v (Lemma "right fixed point", App. C); with exact parents and exact
[Bv] it is the utility gradient of Lemma "Gradient" (App. B) up to the positive
factor <v_i, B v_i>^2 / 2, checked against central finite differences of
Eq. util_new; with B = I and [Bv] = v it equals the projected mu-EigenGame
direction (Prop. "Equivalence to EigenGame Unloaded"); the streamed operators
equal the explicit block matrices of Sec. 1; averaged over many independent
minibatches the update equals the update with population A and B (unbiased
estimates, Sec. 3); Alg. 1 and Alg. 2 with full-batch estimates converge to O1.
LDA (tests/test_oracle_lda.py): streaming every row of a finite set through
`lda_stats_update` gives the between-class scatter of the whole set; with the
batch's own class means `lda_ops` A + B is the batch covariance (law of total
variance); the population problem of Gaussian classes with isotropic shared
covariance reduces to the eigenproblem of the between-class scatter.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# Minibatch operators A_t, B_t (never formed)

def cca_ops(X: np.ndarray, Y: np.ndarray, split: bool = True, eps_B: float = 0.0):
    """CCA minibatch operators (Sec. 1, CCA block form), optional B + eps I (App. G)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    b, dx = X.shape
    nA = b // 2 if split else b
    XA, YA = X[:nA], Y[:nA]
    XB, YB = (X[nA:], Y[nA:]) if split else (X, Y)
    nB = XB.shape[0]

    def Amv(U):
        U = np.asarray(U, dtype=np.float64)
        ux, uy = U[:dx], U[dx:]
        return np.concatenate([XA.T @ (YA @ uy), YA.T @ (XA @ ux)], axis=0) / nA

    def Bmv(U):
        U = np.asarray(U, dtype=np.float64)
        ux, uy = U[:dx], U[dx:]
        out = np.concatenate([XB.T @ (XB @ ux), YB.T @ (YB @ uy)], axis=0) / nB
        return out + eps_B * U

    return Amv, Bmv


def pls_ops(X: np.ndarray, Y: np.ndarray, eps_B: float = 0.0):
    """PLS: A as for CCA over every row, B = I."""
    Amv, _ = cca_ops(X, Y, split=False)
    return Amv, (lambda U: (1.0 + eps_B) * np.asarray(U, dtype=np.float64))


def pca_ops(X: np.ndarray, eps_B: float = 0.0):
    """PCA: A = X^T X / b over every row, B = I (Sec. 1)."""
    X = np.asarray(X, dtype=np.float64)
    b = X.shape[0]

    def Amv(U):
        return X.T @ (X @ np.asarray(U, dtype=np.float64)) / b

    return Amv, (lambda U: (1.0 + eps_B) * np.asarray(U, dtype=np.float64))


def ica_ops(X: np.ndarray, split: bool = True, eps_B: float = 0.0):
    """ICA minibatch operators (Sec. 1, ICA): A = E[<x,x> x x^T] - tr(B) B - 2 B^2, B = E[x x^T].

    A holds products of expectations, so "independent data batches" (Alg. 2) is read with the
    rows in four quarters Q1..Q4 (the last takes the remainder): the kurtosis term of A from Q1,
    tr(B) and the outer B of B^2 from Q2, the B multiplying them from Q3, and B_t from Q4. Every
    product then pairs independent rows and A_t, B_t are unbiased. Without the split every
    term uses every row (the finite-sample pencil of those rows).
    """
    X = np.asarray(X, dtype=np.float64)
    b = X.shape[0]
    if split:
        q = b // 4
        X1, X2, X3, X4 = X[:q], X[q:2 * q], X[2 * q:3 * q], X[3 * q:]
    else:
        X1 = X2 = X3 = X4 = X

    def Bq(Z, U):
        return Z.T @ (Z @ U) / Z.shape[0]

    w1 = np.einsum("rd,rd->r", X1, X1)
    tr2 = np.einsum("rd,rd->", X2, X2) / X2.shape[0]

    def Amv(U):
        U = np.asarray(U, dtype=np.float64)
        B3U = Bq(X3, U)
        return (X1 * w1[:, None]).T @ (X1 @ U) / X1.shape[0] - tr2 * B3U - 2.0 * Bq(X2, B3U)

    def Bmv(U):
        U = np.asarray(U, dtype=np.float64)
        return Bq(X4, U) + eps_B * U

    return Amv, Bmv


def matrix_ops(A: np.ndarray, B: np.ndarray):
    """Exact operators from explicit matrices (full-batch setting)."""
    return (lambda U: A @ U), (lambda U: B @ U)


def lda_stats_update(sums: np.ndarray, counts: np.ndarray, X: np.ndarray, labels: np.ndarray):
    """Running class statistics of LDA: per-class sums of every row seen and counts.

    Reading (the paper names LDA in Sec. 1 without its estimators): the class means
    are the exact cumulative means over all rows seen so far. A step first adds
    every row of its minibatch (both halves), then uses the updated means.
    Returns new (sums, counts); `sums` is C x d, `counts` has C entries.
    """
    sums = np.array(sums, dtype=np.float64, copy=True)
    counts = np.array(counts, dtype=np.float64, copy=True)
    X = np.asarray(X, dtype=np.float64)
    for r in range(X.shape[0]):
        sums[labels[r]] += X[r]
        counts[labels[r]] += 1.0
    return sums, counts


def running_mean_update(sums: np.ndarray, count: float, Z: np.ndarray):
    """Exact running mean of every row seen ("mean estimates are learned", App. H.2.2; the
    methods assume zero-mean data, Sec. 1). Reading: a step first adds every row of its
    minibatch (both halves), then centres those rows by the updated mean. Returns
    (sums, count, mean)."""
    sums = np.asarray(sums, dtype=np.float64) + np.asarray(Z, dtype=np.float64).sum(axis=0)
    count = float(count) + Z.shape[0]
    return sums, count, sums / count


def lda_state(sums: np.ndarray, counts: np.ndarray):
    """Class means mu_c = sums_c / n_c (0 for a class not seen yet) and priors pi_c = n_c / n."""
    counts = np.asarray(counts, dtype=np.float64)
    mean = np.zeros_like(np.asarray(sums, dtype=np.float64))
    seen = counts > 0
    mean[seen] = sums[seen] / counts[seen][:, None]
    return mean, counts / counts.sum()


def lda_ops(X: np.ndarray, labels: np.ndarray, class_mean: np.ndarray,
            class_prior: np.ndarray, split: bool = True, eps_B: float = 0.0):
    """LDA operators given running class means mu_c and priors pi_c (reading, see `form_lda_AB`).

    A U = sum_c pi_c (mu_c - mu)(mu_c - mu)^T U with mu = sum_c pi_c mu_c;
    B U = (1/n_B) sum_r x~_r x~_r^T U with x~_r = x_r - mu_{label r} over the B rows.
    """
    X = np.asarray(X, dtype=np.float64)
    b = X.shape[0]
    nA = b // 2 if split else b
    XB = X[nA:] if split else X
    lB = labels[nA:] if split else labels
    mu = class_prior @ class_mean
    Mc = class_mean - mu[None, :]
    Xt = XB - class_mean[lB]

    def Amv(U):
        U = np.asarray(U, dtype=np.float64)
        return Mc.T @ (class_prior[:, None] * (Mc @ U))

    def Bmv(U):
        U = np.asarray(U, dtype=np.float64)
        return Xt.T @ (Xt @ U) / Xt.shape[0] + eps_B * U

    return Amv, Bmv


# ---------------------------------------------------------------------------
# Rayleigh-Ritz correction of the current players (precision form)

def rayleigh_ritz(V: np.ndarray, S: np.ndarray, Amv, Bmv):
    """Rayleigh-Ritz step in the span of the players, in FP64.

    Solves the k x k pencil (V^T A V) c = lambda (V^T B V) c (A and B estimated on an
    evaluation batch, through the operators), with the Cholesky reduction and Jacobi
    eigensolver of O1 (Prop. "Similar matrices", App. A), and rotates the players into
    the Ritz vectors: V' = V C, [Bv]' = S C (the auxiliary variables follow the same
    linear map), then every column of both is divided by ||v'_i|| (unit sphere).
    Returns (V', S', lam) with lam descending; the columns of V' are ordered by lam
    (signs are those of the k x k eigenvectors, unit Euclidean length in R^k).
    """
    from . import gep
    V = np.asarray(V, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    k = V.shape[1]
    Ak = V.T @ Amv(V)
    Bk = V.T @ Bmv(V)
    Ak = 0.5 * (Ak + Ak.T)
    Bk = 0.5 * (Bk + Bk.T)
    lam, C = gep.gep_topk(Ak, Bk, k)
    Vn = V @ C
    nrm = np.linalg.norm(Vn, axis=0)
    return Vn / nrm[None, :], (S @ C) / nrm[None, :], lam


# ---------------------------------------------------------------------------
# Alg. 2 and Alg. 1

def eg_step(V: np.ndarray, S: np.ndarray, Amv, Bmv, eta: float, gamma: float,
            rho: float, return_parts: bool = False):
    """One iteration of Alg. 2 (M = 1). V, S are d x k: columns v_i and [Bv]_i.

    Returns (V_next, S_next) or, with return_parts, also a dict holding
    AV = A_t V, BV = B_t V and the update directions grad (d x k).
    """
    V = np.asarray(V, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    d, k = V.shape
    AV = Amv(V)          # A_t v_i for every player
    BV = Bmv(V)          # B_t v_i for every player
    grad = np.zeros_like(V)
    for i in range(k):
        vi = V[:, i]
        Avi = AV[:, i]
        Bvi = BV[:, i]
        vBv = vi @ Bvi
        vAv = vi @ Avi
        rewards = vBv * Avi - vAv * Bvi
        penalties = np.zeros(d)
        for j in range(i):
            denom = np.sqrt(max(V[:, j] @ S[:, j], rho))  # y_j = v_j / denom
            Byj = S[:, j] / denom
            # v_i^T A_t y_j as Alg. 2 writes it (A_t y_j = A_t v_j / denom); an estimate A_t
            # need not be symmetric (ICA's products of independent quarters are not)
            vAy = vi @ AV[:, j] / denom
            penalties += vAy * (vBv * Byj - (vi @ Byj) * Bvi)
        grad[:, i] = rewards - penalties
    Vp = V + eta * grad
    V_next = Vp / np.linalg.norm(Vp, axis=0, keepdims=True)
    S_next = S + gamma * (BV - S)
    if return_parts:
        return V_next, S_next, {"AV": AV, "BV": BV, "grad": grad}
    return V_next, S_next


def eg_step_machines(V: np.ndarray, S: np.ndarray, machine_ops, eta: float, gamma: float, rho: float):
    """One iteration of Alg. 2 with M = len(machine_ops) machines.

    Machine m holds its own minibatch estimates (A_tm, B_tm) (the operators of its shard) and
    forms, from the shared state of step t, the update direction grad_im of every player
    (rewards minus penalties, Eq. update) and the auxiliary increment B_tm v_i - [Bv]_i; both
    are averaged over the machines, then the player step with the retraction and the
    auxiliary step follow, as Alg. 2 writes them. Returns (V_next, S_next).
    """
    V = np.asarray(V, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    M = len(machine_ops)
    grad = np.zeros_like(V)
    inc = np.zeros_like(S)
    for Amv, Bmv in machine_ops:
        _, _, parts = eg_step(V, S, Amv, Bmv, 0.0, 0.0, rho, return_parts=True)
        grad += parts["grad"] / M
        inc += (parts["BV"] - S) / M
    Vp = V + eta * grad
    return Vp / np.linalg.norm(Vp, axis=0, keepdims=True), S + gamma * inc


def smooth_denominator(z: np.ndarray, rho: float, nu: float) -> np.ndarray:
    """[<v, B v>]_j of Alg. 3: exp(log rho + (log nu - log rho) sigmoid(z_j)), in (rho, nu)."""
    z = np.asarray(z, dtype=np.float64)
    sig = 1.0 / (1.0 + np.exp(-z))
    return np.exp(np.log(rho) + (np.log(nu) - np.log(rho)) * sig)


def eg_step_variant(V: np.ndarray, S: np.ndarray, Amv, Bmv, eta: float, gamma: float, rho: float,
                    adam: dict | None = None, smooth: dict | None = None, return_parts: bool = False):
    """One iteration of Alg. 2 (M = 1) with the two variants the paper describes.

    smooth = {"z": z (k,), "nu": nu}: Alg. 3 (App. E.2). Player j's denominator is
    s_j = exp(log rho + (log nu - log rho) sigmoid(z_j)) instead of max(<v_j, [Bv]_j>, rho);
    every player also takes z_i <- z_i + gamma (<v_i, [Bv]_i> - s_i) s_i (log nu - log rho)
    sigmoid(z_i) (1 - sigmoid(z_i)), with the state of step t.
    adam = {"m": m, "s": s (d x k), "t": t (steps taken so far), "b1", "b2", "eps"}: the player
    step of App. H.2.2 ("Adam on v_i"): with the update direction g_i of the step,
    m_i <- b1 m_i + (1 - b1) g_i, s_i <- b2 s_i + (1 - b2) g_i^2 (elementwise),
    v_i' = v_i + eta (m_i / (1 - b1^(t+1))) / (sqrt(s_i / (1 - b2^(t+1))) + eps), then v_i' / |v_i'|.
    Reading: Adam replaces the plain step v_i + eta g_i of Alg. 2 and the retraction stays.
    Returns (V_next, S_next, state) with state = {"adam": ..., "smooth": ...} (new dicts), and
    with return_parts also a dict with AV, BV and grad.
    """
    V = np.asarray(V, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    d, k = V.shape
    AV = Amv(V)
    BV = Bmv(V)
    if smooth is not None:
        den = smooth_denominator(smooth["z"], rho, smooth["nu"])
    else:
        den = np.array([max(V[:, j] @ S[:, j], rho) for j in range(k)])
    grad = np.zeros_like(V)
    for i in range(k):
        vi, Avi, Bvi = V[:, i], AV[:, i], BV[:, i]
        vBv = vi @ Bvi
        vAv = vi @ Avi
        rewards = vBv * Avi - vAv * Bvi
        penalties = np.zeros(d)
        for j in range(i):
            Byj = S[:, j] / np.sqrt(den[j])
            penalties += (vi @ AV[:, j] / np.sqrt(den[j])) * (vBv * Byj - (vi @ Byj) * Bvi)
        grad[:, i] = rewards - penalties
    state = {}
    if adam is not None:
        b1, b2, eps, t = adam["b1"], adam["b2"], adam["eps"], int(adam["t"]) + 1
        m = b1 * np.asarray(adam["m"], np.float64) + (1.0 - b1) * grad
        s = b2 * np.asarray(adam["s"], np.float64) + (1.0 - b2) * grad * grad
        step = (m / (1.0 - b1 ** t)) / (np.sqrt(s / (1.0 - b2 ** t)) + eps)
        state["adam"] = {"m": m, "s": s, "t": t, "b1": b1, "b2": b2, "eps": eps}
    else:
        step = grad
    Vp = V + eta * step
    V_next = Vp / np.linalg.norm(Vp, axis=0, keepdims=True)
    S_next = S + gamma * (BV - S)
    if smooth is not None:
        z = np.asarray(smooth["z"], np.float64)
        nu = smooth["nu"]
        sig = 1.0 / (1.0 + np.exp(-z))
        c = np.array([V[:, i] @ S[:, i] for i in range(k)])
        gz = (c - den) * den * (np.log(nu) - np.log(rho)) * sig * (1.0 - sig)
        state["smooth"] = {"z": z + gamma * gz, "nu": nu}
    if return_parts:
        return V_next, S_next, state, {"AV": AV, "BV": BV, "grad": grad}
    return V_next, S_next, state


def alg1_step(V: np.ndarray, A: np.ndarray, B: np.ndarray, eta: float) -> np.ndarray:
    """One iteration of the deterministic algorithm (Alg. 1) with exact A and B."""
    V = np.asarray(V, dtype=np.float64)
    d, k = V.shape
    AV = A @ V
    BV = B @ V
    grad = np.zeros_like(V)
    for i in range(k):
        vi = V[:, i]
        rewards = (vi @ BV[:, i]) * AV[:, i] - (vi @ AV[:, i]) * BV[:, i]
        penalties = np.zeros(d)
        for j in range(i):
            nj = np.sqrt(V[:, j] @ BV[:, j])
            yj = V[:, j] / nj
            Byj = BV[:, j] / nj
            penalties += (AV[:, i] @ yj) * ((vi @ BV[:, i]) * Byj - (vi @ Byj) * BV[:, i])
        grad[:, i] = rewards - penalties
    Vp = V + eta * grad
    return Vp / np.linalg.norm(Vp, axis=0, keepdims=True)


def utility(V: np.ndarray, i: int, A: np.ndarray, B: np.ndarray) -> float:
    """u_i(v_i | v_{j<i}) of Eq. util_new: generalized Rayleigh quotient minus penalties."""
    vi = V[:, i]
    vBv = vi @ B @ vi
    u = (vi @ A @ vi) / vBv
    for j in range(i):
        vj = V[:, j]
        vjBvj = vj @ B @ vj
        u -= (vj @ A @ vj) * (vi @ B @ vj) ** 2 / (vjBvj ** 2 * vBv)
    return float(u)


# ---------------------------------------------------------------------------
# Step sizes (App. H.2.2)

def schedule_eta(t: int, eta0: float, schedule: int, t_c: int = 0, T: int = 1,
                 eta_T: float = 0.0) -> float:
    """Player step size eta_t for iteration t = 1, 2, ...

    schedule 0: constant eta0.
    schedule 1: eta0 up to t_c, then proportional to 1/(t + Delta), reaching eta_T at T.
    schedule 2: linear warm-up eta0 t / t_c up to t_c, then the same harmonic decay
                (the schedule of App. H.2.2).
    Delta solves eta0 (t_c + Delta) / (T + Delta) = eta_T.
    """
    if schedule == 0:
        return float(eta0)
    delta = (eta_T * T - eta0 * t_c) / (eta0 - eta_T)
    if t <= t_c:
        return float(eta0 if schedule == 1 else eta0 * t / t_c)
    return float(eta0 * (t_c + delta) / (t + delta))
