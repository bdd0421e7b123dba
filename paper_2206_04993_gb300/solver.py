"""A small object wrapper around the C handle (marshalling only)."""
from __future__ import annotations

import numpy as np

from . import sgep as _s


class Solver:
    """Owns one sgep handle. Inputs are torch CUDA tensors (row-major samples)."""

    def __init__(self, **cfg):
        self.cfg = _s.sgep_config_default(**cfg)
        self.h = _s.sgep_init(self.cfg)
        self.d = self.cfg.d_x + self.cfg.d_y
        self.k = self.cfg.k

    def close(self):
        if self.h:
            _s.sgep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _cur_stream():
        import torch
        return torch.cuda.current_stream().cuda_stream

    def step(self, X, Y=None, b=None, labels=None, sx=None, sy=None):
        """One step on device rows X (and Y); LDA also takes int32 device labels, FP8 rows
        their per-row scales sx (and sy)."""
        _s.sgep_step(self.h, X, Y, labels, X.shape[0] if b is None else b, self._cur_stream(), sx, sy)

    def step_many(self, X, Y, b, nsteps, labels=None, sx=None, sy=None):
        _s.sgep_step_many(self.h, X, Y, b, nsteps, labels, self._cur_stream(), sx, sy)

    def sync(self):
        _s.sgep_sync(self.h, self._cur_stream())

    def V(self) -> np.ndarray:
        out = np.empty((self.d, self.k), dtype=np.float32)
        _s.sgep_get_V(self.h, out, False, self._cur_stream())
        return out

    def S(self) -> np.ndarray:
        out = np.empty((self.d, self.k), dtype=np.float32)
        _s.sgep_get_S(self.h, out, False, self._cur_stream())
        return out

    def set_V(self, V, S=None):
        V = np.ascontiguousarray(V, dtype=np.float32)
        if S is None:
            _s.sgep_set_V(self.h, V, False, self._cur_stream())
        else:
            S = np.ascontiguousarray(S, dtype=np.float32)
            _s.sgep_set_VS(self.h, V, S, False, self._cur_stream())

    def eigenvalues(self, X, Y=None, labels=None, sx=None, sy=None) -> np.ndarray:
        out = np.empty(self.k, dtype=np.float64)
        _s.sgep_get_eigenvalues(self.h, X, Y, X.shape[0], out, labels, self._cur_stream(), sx, sy)
        return out

    def rayleigh_ritz(self, X, Y=None, labels=None, sx=None, sy=None) -> np.ndarray:
        """Rotate the players into the Ritz vectors of their span on rows (X, Y); Ritz values."""
        out = np.empty(self.k, dtype=np.float64)
        _s.sgep_rayleigh_ritz(self.h, X, Y, X.shape[0], out, labels, self._cur_stream(), sx, sy)
        return out

    def set_rr_every(self, every, X=None, Y=None, labels=None, sx=None, sy=None):
        """Rayleigh-Ritz correction on the evaluation rows (X, Y) after every `every` steps
        (0 removes it); the rows must stay alive and unchanged while it is set."""
        n = 0 if X is None else X.shape[0]
        self._rr_rows = (X, Y, labels, sx, sy) if every else None  # keep them alive
        _s.sgep_set_rr_every(self.h, every, X, Y, n, labels, sx, sy)

    def products(self):
        AV = np.empty((self.d, self.k), dtype=np.float32)
        BV = np.empty((self.d, self.k), dtype=np.float32)
        _s.sgep_debug_products(self.h, AV, BV)
        return AV, BV

    def update_terms(self):
        grad = np.empty((self.d, self.k), dtype=np.float32)
        terms = np.empty(2 * self.k * self.k + self.k, dtype=np.float64)
        _s.sgep_debug_update(self.h, grad, terms)
        k = self.k
        return grad, terms[:k * k].reshape(k, k), terms[k * k:2 * k * k].reshape(k, k), terms[2 * k * k:]

    @property
    def t(self) -> int:
        return _s.sgep_step_count(self.h)

    @property
    def launches(self) -> int:
        return _s.sgep_launch_count(self.h)

    @property
    def path(self) -> int:
        return _s.sgep_path(self.h)

    def state(self) -> bytes:
        return _s.sgep_get_state(self.h)

    def load_state(self, blob: bytes):
        _s.sgep_set_state(self.h, blob)


class Batch:
    """Many Solvers (generic path) advanced by one batched launch per step."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.b = _s.sgep_batch_create([x.h for x in self.solvers])

    def close(self):
        if getattr(self, "b", None) is not None:
            _s.sgep_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream():
        import torch
        return torch.cuda.current_stream().cuda_stream

    def step(self, Xs, Ys=None, rows=None, labels=None, sx=None, sy=None):
        rows = [x.shape[0] for x in Xs] if rows is None else rows
        _s.sgep_batch_step(self.b, Xs, Ys, rows, labels, sx, sy, self._stream())

    def sync(self):
        _s.sgep_batch_sync(self.b, self._stream())

    def configure(self, mode=-1, blocks_per_sm=0, chunk_cap=0, rows_cap=0, use_graph=-1):
        _s.sgep_batch_configure(self.b, mode, blocks_per_sm, chunk_cap, rows_cap, use_graph)

    def config(self):
        return _s.sgep_batch_get_config(self.b)

    def autotune(self, Xs, Ys=None, rows=None, labels=None, sx=None, sy=None, reps=3):
        rows = [x.shape[0] for x in Xs] if rows is None else rows
        return _s.sgep_batch_autotune(self.b, Xs, Ys, rows, labels, sx, sy, reps)

    def launches(self) -> int:
        return _s.sgep_batch_launch_count(self.b)


class WarmStart:
    """Sketch-to-players network (hand-written CUDA kernels): rows of the sketch
    Z^T (Z Omega) / n of a first minibatch map to rows of an initial V."""

    def __init__(self, m=16, k=16, seed=0):
        self.m, self.k = m, k
        self.h = _s.sgep_mlp_create(m, k, seed)
        self.P = _s.sgep_mlp_param_count(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            _s.sgep_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream():
        import torch
        return torch.cuda.current_stream().cuda_stream

    def params(self) -> np.ndarray:
        out = np.empty(self.P, dtype=np.float32)
        _s.sgep_mlp_get_params(self.h, out)
        return out

    def set_params(self, p):
        _s.sgep_mlp_set_params(self.h, np.ascontiguousarray(p, dtype=np.float32))

    @staticmethod
    def sketch(X, Y, omega, dtype=0):
        """Device sketch (d x m float32) of device rows X (and Y) with device Omega (d x m)."""
        import torch
        d = X.shape[1] + (0 if Y is None else Y.shape[1])
        out = torch.empty((d, omega.shape[1]), dtype=torch.float32, device=X.device)
        _s.sgep_sketch(X, Y, dtype, X.shape[0], X.shape[1], 0 if Y is None else Y.shape[1], omega, omega.shape[1],
                       out, WarmStart._stream())
        return out

    def forward(self, S):
        import torch
        out = torch.empty((S.shape[0], self.k), dtype=torch.float32, device=S.device)
        _s.sgep_mlp_forward(self.h, S, S.shape[0], out, self._stream())
        return out

    def loss_grad(self, S, V, seg, grads=False):
        g = np.empty(self.P, dtype=np.float32) if grads else None
        loss = _s.sgep_mlp_loss_grad(self.h, S, V, seg, len(seg) - 1, g, self._stream())
        return (loss, g) if grads else loss

    def adam_step(self, lr):
        _s.sgep_mlp_adam_step(self.h, lr, self._stream())
