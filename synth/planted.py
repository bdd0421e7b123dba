"""Planted data models for the symmetric generalized eigenproblem workloads.

All randomness comes from numpy's Philox-4x32-10 counter-based generator
(Salmon et al., SC'11), keyed by (seed, stream). A stream id separates the
model parameters, the initial player vectors and each minibatch, so any
minibatch can be regenerated on its own.

Models (all zero-mean, matching the paper's zero-mean assumption, Sec. 1):

* PlantedCCA: x = Q_x diag(s) z + sigma e_x, y = Q_y diag(s) z + sigma e_y with
  z ~ N(0, I_r), Q_x, Q_y orthonormal columns (QR of a Gaussian matrix). With
  s_l^2 = sigma^2 rho_l / (1 - rho_l) the canonical correlations are exactly
  rho_l (used for the 4- and 16-player CCA workloads).
* PlantedLowRankCCA: x = D_x^{1/2} g_x + W_x z, y = D_y^{1/2} g_y + W_y z with a
  power-law diagonal D (D_ii proportional to i^-alpha) and m planted shared
  directions (the activation-like workload, d_x = d_y = 16384).
* PCA: x = Q diag(sqrt(spectrum)) z + sigma e.
* LDA: C Gaussian classes with means mu_c and a shared within-class covariance.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Stream ids: the key of each Philox generator is (seed, stream).
_STREAM_MODEL = 1
_STREAM_INIT = 2
_STREAM_FINITE = 3
_STREAM_INDEX_BASE = 1 << 20
_STREAM_ROWS_BASE = 1 << 40


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.array([seed, stream], dtype=np.uint64)))


def _orthonormal(rng: np.random.Generator, d: int, r: int) -> np.ndarray:
    q, rr = np.linalg.qr(rng.standard_normal((d, r)))
    return q * np.sign(np.diag(rr))[None, :]


@dataclass
class PlantedCCA:
    Qx: np.ndarray      # d_x x r, orthonormal columns
    Qy: np.ndarray      # d_y x r, orthonormal columns
    s: np.ndarray       # r latent scales
    sigma: float        # isotropic noise level
    rhos: np.ndarray    # the planted canonical correlations (input, for reference)
    seed: int

    @property
    def d_x(self) -> int:
        return self.Qx.shape[0]

    @property
    def d_y(self) -> int:
        return self.Qy.shape[0]

    @property
    def Wx(self) -> np.ndarray:
        return self.Qx * self.s[None, :]

    @property
    def Wy(self) -> np.ndarray:
        return self.Qy * self.s[None, :]


@dataclass
class PlantedLowRankCCA:
    Dx: np.ndarray      # d_x diagonal noise variances
    Dy: np.ndarray
    Wx: np.ndarray      # d_x x m
    Wy: np.ndarray      # d_y x m
    seed: int

    @property
    def d_x(self) -> int:
        return self.Wx.shape[0]

    @property
    def d_y(self) -> int:
        return self.Wy.shape[0]


def planted_cca(d_x: int, d_y: int, rhos, sigma: float = 0.5, seed: int = 0) -> PlantedCCA:
    rhos = np.asarray(rhos, dtype=np.float64)
    rng = _rng(seed, _STREAM_MODEL)
    r = rhos.size
    Qx = _orthonormal(rng, d_x, r)
    Qy = _orthonormal(rng, d_y, r)
    s = np.sqrt(sigma * sigma * rhos / (1.0 - rhos))
    return PlantedCCA(Qx, Qy, s, float(sigma), rhos, seed)


def planted_lowrank_cca(d_x: int, d_y: int, m: int = 64, alpha: float = 1.0,
                        target_rhos=None, seed: int = 0) -> PlantedLowRankCCA:
    """Activation-like CCA model: power-law per-coordinate noise plus m shared directions.

    D_ii = i^-alpha (i = 1..d). The shared directions are W = Q diag(w) with Q a
    random orthonormal d x m matrix. For such Q, H = W^T D^-1 W is close to
    diag(w^2) mean(1/D), and the canonical correlations are close to
    h_l / (1 + h_l); w is set from `target_rhos` (default 0.95 down to 0.3)
    through that approximation. The exact correlations follow from the model
    and are computed by the oracle's closed form, not taken from here.
    """
    rng = _rng(seed, _STREAM_MODEL)
    Dx = np.arange(1, d_x + 1, dtype=np.float64) ** (-alpha)
    Dy = np.arange(1, d_y + 1, dtype=np.float64) ** (-alpha)
    if target_rhos is None:
        target_rhos = np.linspace(0.95, 0.3, m)
    h = np.asarray(target_rhos, dtype=np.float64)
    h = h / (1.0 - h)
    wx = np.sqrt(h / np.mean(1.0 / Dx))
    wy = np.sqrt(h / np.mean(1.0 / Dy))
    Wx = _orthonormal(rng, d_x, m) * wx[None, :]
    Wy = _orthonormal(rng, d_y, m) * wy[None, :]
    return PlantedLowRankCCA(Dx, Dy, Wx, Wy, seed)


def planted_pca(d: int, spectrum, sigma: float = 0.1, seed: int = 0):
    rng = _rng(seed, _STREAM_MODEL)
    spectrum = np.asarray(spectrum, dtype=np.float64)
    Q = _orthonormal(rng, d, spectrum.size)
    return {"Q": Q, "spectrum": spectrum, "sigma": float(sigma), "seed": seed}


def planted_lda(d: int, n_classes: int = 10, sigma_b: float = 1.0, seed: int = 0, rotate: bool = True):
    """C Gaussian classes, equal priors, means N(0, sigma_b^2 I), shared covariance L L^T
    (L = rotation x diag(1..0.5); rotate=False keeps L diagonal, for large d)."""
    rng = _rng(seed, _STREAM_MODEL)
    means = sigma_b * rng.standard_normal((n_classes, d))
    means -= means.mean(axis=0, keepdims=True)   # zero overall mean
    scales = np.linspace(1.0, 0.5, d)
    L = _orthonormal(rng, d, d) * scales[None, :] if rotate else np.diag(scales)
    return {"means": means, "L": L, "scales": scales, "seed": seed}


def draw_rows(model, n: int, batch: int, dtype=np.float64):
    """Rows of minibatch number `batch` (n paired samples) from a CCA model."""
    rng = _rng(model.seed, _STREAM_ROWS_BASE + batch)
    if isinstance(model, PlantedCCA):
        z = rng.standard_normal((n, model.s.size))
        X = z @ model.Wx.T + model.sigma * rng.standard_normal((n, model.d_x))
        Y = z @ model.Wy.T + model.sigma * rng.standard_normal((n, model.d_y))
    else:
        z = rng.standard_normal((n, model.Wx.shape[1]))
        X = z @ model.Wx.T + rng.standard_normal((n, model.d_x)) * np.sqrt(model.Dx)[None, :]
        Y = z @ model.Wy.T + rng.standard_normal((n, model.d_y)) * np.sqrt(model.Dy)[None, :]
    return X.astype(dtype), Y.astype(dtype)


def draw_pca_rows(model, n: int, batch: int, dtype=np.float64):
    rng = _rng(model["seed"], _STREAM_ROWS_BASE + batch)
    z = rng.standard_normal((n, model["spectrum"].size)) * np.sqrt(model["spectrum"])[None, :]
    X = z @ model["Q"].T + model["sigma"] * rng.standard_normal((n, model["Q"].shape[0]))
    return X.astype(dtype)


def draw_lda_rows(model, n: int, batch: int, dtype=np.float64):
    rng = _rng(model["seed"], _STREAM_ROWS_BASE + batch)
    C, d = model["means"].shape
    labels = rng.integers(0, C, size=n).astype(np.int32)
    X = model["means"][labels] + rng.standard_normal((n, d)) @ model["L"].T
    return X.astype(dtype), labels


# Source laws of the ICA model: unit variance, known excess kurtosis E[s^4] - 3.
#   "rademacher": +-1 (kurtosis -2); "uniform": U[-sqrt 3, sqrt 3] (-1.2); "laplace": Laplace
#   with scale 1/sqrt 2 (3); "sparse": 0 w.p. 3/4, +-2 w.p. 1/8 each (1); "gauss": N(0, 1) (0).
ICA_KURTOSIS = {"rademacher": -2.0, "uniform": -1.2, "laplace": 3.0, "sparse": 1.0, "gauss": 0.0}


def planted_ica(d: int, laws, seed: int = 0, cond: float = 3.0):
    """Linear mixture x = M s of d independent unit-variance sources with the given laws
    (stand-in for the mixed signals of the ICA experiment); M has singular values from 1 to
    `cond` between random rotations."""
    rng = _rng(seed, _STREAM_MODEL)
    laws = list(laws)
    assert len(laws) == d
    U = _orthonormal(rng, d, d)
    W = _orthonormal(rng, d, d)
    M = (U * np.linspace(1.0, cond, d)[None, :]) @ W.T
    return {"M": M, "laws": laws, "kurtosis": np.array([ICA_KURTOSIS[l] for l in laws]), "seed": seed}


def _source(rng, law: str, n: int) -> np.ndarray:
    if law == "rademacher":
        return rng.choice([-1.0, 1.0], size=n)
    if law == "uniform":
        return rng.uniform(-np.sqrt(3.0), np.sqrt(3.0), size=n)
    if law == "laplace":
        return rng.laplace(0.0, 1.0 / np.sqrt(2.0), size=n)
    if law == "sparse":
        u = rng.uniform(size=n)
        return np.where(u < 0.125, -2.0, np.where(u < 0.25, 2.0, 0.0))
    return rng.standard_normal(n)


def draw_ica_rows(model, n: int, batch: int, dtype=np.float64):
    """Rows x = M s of minibatch number `batch`."""
    rng = _rng(model["seed"], _STREAM_ROWS_BASE + batch)
    Ssrc = np.stack([_source(rng, law, n) for law in model["laws"]], axis=1)
    return (Ssrc @ model["M"].T).astype(dtype)


def random_unit_columns(d: int, k: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """Initial strategies: v_i ~ N(0, I_d) then scaled to unit norm (Alg. 2 init)."""
    V = _rng(seed, _STREAM_INIT).standard_normal((d, k))
    V /= np.sqrt(np.sum(V * V, axis=0, keepdims=True))
    return V.astype(dtype)


def finite_dataset_indices(n_total: int, b: int, step: int, seed: int = 0) -> np.ndarray:
    """Indices of minibatch `step`, drawn with replacement from a finite dataset."""
    return _rng(seed, _STREAM_INDEX_BASE + step).integers(0, n_total, size=b)


# ---------------------------------------------------------------------------
# The named workloads. Each returns a plain dict of shapes and hyperparameters
# plus the planted model.

def config_c1(seed: int = 0):
    """Plain CCA, d_x = d_y = 32, k = 4, a finite set of 10,000 paired rows, b = 256."""
    rhos = np.array([0.9, 0.8, 0.7, 0.6, 0.5, 0.4, 0.3, 0.2])
    model = planted_cca(32, 32, rhos, sigma=0.5, seed=seed)
    X, Y = draw_rows(model, 10_000, batch=_STREAM_FINITE)
    return {"name": "cca_d64_k4_b256", "model": model, "X": X, "Y": Y, "k": 4, "b": 256,
            # hold 0.3 for 300 steps, then harmonic down to 0.3 * 0.012 at step 2000 (the best
            # point of a sweep of eta0, t_c and eta_T / eta0 on the oracle: error floor ~8.6e-4)
            "steps": 2000, "eta0": 0.3, "gamma0": 0.3, "rho": 1e-6,
            "schedule": 1, "t_c": 300, "T": 2000, "eta_T": 0.3 * 0.012}


def config_c2(seed: int = 0):
    """Plain CCA, d_x = d_y = 512, k = 16, b = 1024, latent dim 32, rho 0.95..0.3."""
    rhos = np.linspace(0.95, 0.3, 32)
    model = planted_cca(512, 512, rhos, sigma=0.5, seed=seed)
    # harmonic step eta_t = 0.2 (1 + 400) / (t + 400) (tuned: the paper gives none for this size)
    return {"name": "cca_d1024_k16_b1024", "model": model, "k": 16, "b": 1024,
            "n_samples": 1_000_000, "eta0": 0.2, "gamma0": 0.3, "rho": 1e-6,
            "schedule": 1, "t_c": 1, "T": 20000, "eta_T": 0.2 * 401.0 / 20400.0}


def config_c3(seed: int = 0):
    """Activation-like CCA, d_x = d_y = 16384, k = 32, b = 4096, 64 planted directions."""
    model = planted_lowrank_cca(16384, 16384, m=64, alpha=1.0, seed=seed)
    return {"name": "cca_d32768_k32_b4096", "model": model, "k": 32, "b": 4096,
            "n_samples": 10_000_000, "eta0": 0.3, "gamma0": 0.3, "rho": 1e-6,
            "schedule": 1, "t_c": 100, "T": 2442, "eta_T": 0.3 * 120.0 / 2462.0}


# ---------------------------------------------------------------------------
# FP8 e4m3 rows with one scale per row (input encoding of the precision form)

def _e4m3_table():
    """All finite non-negative e4m3 values, indexed by code 0..0x7E (sign bit clear)."""
    vals = []
    for code in range(0x7F):
        e, m = code >> 3, code & 7
        vals.append((m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(vals)


def quantize_e4m3_rows(X):
    """Per-row scale s_r = max|x_r| / 448 (1 for an all-zero row) and the e4m3 codes of
    x_r / s_r rounded to the nearest value (ties to the even code). Returns (codes uint8,
    scales float32); the represented rows are s_r * e4m3(codes)."""
    X = np.asarray(X, dtype=np.float64)
    scales = np.max(np.abs(X), axis=1) / 448.0
    scales[scales == 0] = 1.0
    scales = scales.astype(np.float32)
    Z = X / scales.astype(np.float64)[:, None]
    table = _e4m3_table()
    a = np.minimum(np.abs(Z), 448.0)
    hi = np.clip(np.searchsorted(table, a, side="left"), 0, len(table) - 1)
    lo = np.clip(hi - 1, 0, len(table) - 1)
    dlo, dhi = a - table[lo], table[hi] - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    code = np.where(pick_hi, hi, lo).astype(np.uint8)
    code = np.where(Z < 0, code | 0x80, code).astype(np.uint8)
    return code, scales


def config_c4(seed: int = 0, n_instances: int = 64):
    """Batching workload: independent instances, even ones CCA (d uniform in 64..4096,
    d_x = d_y = d / 2, planted with 16 latent directions, correlations 0.9..0.3) and odd
    ones LDA (10 Gaussian classes, d uniform in 64..4096, diagonal within-class covariance);
    k uniform in 4..32, clamped to 9 for LDA (rank of the between-class scatter); b = 512."""
    rng = _rng(seed, _STREAM_MODEL + 7)
    out = []
    for i in range(n_instances):
        d = int(rng.integers(64, 4097))
        k = int(rng.integers(4, 33))
        if i % 2 == 0:
            dx = max(16, d // 2)
            out.append({"kind": "cca", "d_x": dx, "d_y": dx, "k": min(k, dx), "b": 512,
                        "model": planted_cca(dx, dx, np.linspace(0.9, 0.3, 16), sigma=0.5, seed=seed * 1000 + i)})
        else:
            out.append({"kind": "lda", "d_x": d, "d_y": 0, "k": min(k, 9), "b": 512, "n_classes": 10,
                        "model": planted_lda(d, n_classes=10, seed=seed * 1000 + i, rotate=False)})
    return out


def config_c5(seed: int = 0, d_x: int = 1024, k: int = 16, latent: int = 16, n_theta: int = 8,
              spread: float = 0.3):
    """Warm-start family: CCA instances whose mixing matrices are a fixed smooth function
    of theta ~ U[-1, 1]^n_theta: Q_view(theta) = orthonormalise(W0 + spread * sum_m theta_m W_m)
    (d_x = d_y, `latent` planted directions, correlations 0.9..0.3, noise 0.5). Returns a
    function theta -> PlantedCCA, a sampler of theta, and the sketch matrix Omega (d x 16)."""
    rng = _rng(seed, _STREAM_MODEL + 11)
    d = 2 * d_x
    W0 = [rng.standard_normal((d_x, latent)) for _ in range(2)]
    Wm = [[rng.standard_normal((d_x, latent)) for _ in range(n_theta)] for _ in range(2)]
    rhos = np.linspace(0.9, 0.3, latent)
    s = np.sqrt(0.25 * rhos / (1.0 - rhos))
    omega = rng.standard_normal((d, 16))

    def model(theta):
        Q = []
        for v in range(2):
            M = W0[v] + spread * sum(theta[m] * Wm[v][m] for m in range(n_theta))
            q, r = np.linalg.qr(M)
            Q.append(q * np.sign(np.diag(r))[None, :])
        return PlantedCCA(Q[0], Q[1], s.copy(), 0.5, rhos.copy(), seed)

    def thetas(n, stream):
        return _rng(seed, _STREAM_MODEL + 100 + stream).uniform(-1.0, 1.0, size=(n, n_theta))

    return {"model": model, "thetas": thetas, "omega": omega, "d_x": d_x, "k": k, "latent": latent}
