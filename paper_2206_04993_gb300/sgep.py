"""ctypes binding of libsgep (include/sgep.h): the same entry points, argument
marshalling only. Every step of the method runs in the library's CUDA kernels;
there is no Python or CPU fallback. If libsgep.so is missing the first call
raises RuntimeError.

Tensors are passed as raw pointers: `data_ptr()` of torch tensors (device
memory) or numpy arrays (host memory), and streams as
`torch.cuda.current_stream().cuda_stream`.
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsgep.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "sgep.h")

SGEP_OK, SGEP_EINVAL, SGEP_ENOMEM, SGEP_ECUDA = 0, -1, -2, -3
SGEP_ETIMEOUT, SGEP_ENONFINITE, SGEP_ELAUNCH, SGEP_ESTATE, SGEP_ENOTSUP = -4, -5, -6, -7, -8
SGEP_PCA, SGEP_CCA, SGEP_PLS, SGEP_LDA, SGEP_ICA = 0, 1, 2, 3, 4
SGEP_F32, SGEP_BF16, SGEP_FP8E4M3 = 0, 1, 2
SGEP_SCHED_CONST, SGEP_SCHED_HOLD_HARMONIC, SGEP_SCHED_WARMUP_HARMONIC = 0, 1, 2
SGEP_PATH_AUTO, SGEP_PATH_GENERIC, SGEP_PATH_CLUSTER, SGEP_PATH_TC = 0, 1, 2, 3
SGEP_OPT_SGD, SGEP_OPT_ADAM = 0, 1
SGEP_ALG2, SGEP_ALG3 = 0, 1


class sgep_config(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("dtype", ctypes.c_int32),
        ("d_x", ctypes.c_int64), ("d_y", ctypes.c_int64),
        ("k", ctypes.c_int32), ("n_classes", ctypes.c_int32),
        ("eta0", ctypes.c_float), ("gamma0", ctypes.c_float),
        ("rho", ctypes.c_float), ("eps_B", ctypes.c_float),
        ("schedule", ctypes.c_int32), ("split_AB", ctypes.c_int32),
        ("t_c", ctypes.c_int64), ("T", ctypes.c_int64), ("eta_T", ctypes.c_float),
        ("path", ctypes.c_int32), ("seed", ctypes.c_uint64), ("max_b", ctypes.c_int64),
        ("debug", ctypes.c_int32), ("optimizer", ctypes.c_int32), ("adam_b1", ctypes.c_float),
        ("adam_b2", ctypes.c_float), ("adam_eps", ctypes.c_float), ("variant", ctypes.c_int32),
        ("nu", ctypes.c_float), ("center", ctypes.c_int32),
        ("machines", ctypes.c_int32), ("reserved0", ctypes.c_int32),
    ]


class SgepError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


_P = ctypes.c_void_p
_SIGS = {
    "sgep_config_default": (ctypes.c_int, [ctypes.POINTER(sgep_config)]),
    "sgep_init": (ctypes.c_int, [ctypes.POINTER(sgep_config), ctypes.POINTER(_P)]),
    "sgep_destroy": (ctypes.c_int, [_P]),
    "sgep_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int64, _P]),
    "sgep_step_many": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int64, _P]),
    "sgep_sync": (ctypes.c_int, [_P, _P]),
    "sgep_get_V": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "sgep_get_S": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "sgep_set_V": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "sgep_set_VS": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "sgep_get_eigenvalues": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int64, _P, _P]),
    "sgep_rayleigh_ritz": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int64, _P, _P]),
    "sgep_set_rr_every": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P, _P, ctypes.c_int64]),
    "sgep_batch_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "sgep_batch_destroy": (ctypes.c_int, [_P]),
    "sgep_batch_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "sgep_batch_sync": (ctypes.c_int, [_P, _P]),
    "sgep_batch_configure": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int]),
    "sgep_batch_get_config": (ctypes.c_int, [_P, _P]),
    "sgep_batch_autotune": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int, _P]),
    "sgep_batch_launch_count": (ctypes.c_int64, [_P]),
    "sgep_sketch": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P,
                                   ctypes.c_int, _P, _P]),
    "sgep_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "sgep_mlp_destroy": (ctypes.c_int, [_P]),
    "sgep_mlp_param_count": (ctypes.c_int, [_P]),
    "sgep_mlp_get_params": (ctypes.c_int, [_P, _P]),
    "sgep_mlp_set_params": (ctypes.c_int, [_P, _P]),
    "sgep_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "sgep_mlp_loss_grad": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, _P, _P, _P]),
    "sgep_mlp_adam_step": (ctypes.c_int, [_P, ctypes.c_float, _P]),
    "sgep_get_state": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "sgep_set_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "sgep_step_count": (ctypes.c_int64, [_P]),
    "sgep_eta_at": (ctypes.c_double, [_P, ctypes.c_int64]),
    "sgep_path": (ctypes.c_int, [_P]),
    "sgep_launch_count": (ctypes.c_int64, [_P]),
    "sgep_debug_products": (ctypes.c_int, [_P, _P, _P]),
    "sgep_debug_update": (ctypes.c_int, [_P, _P, _P]),
    "sgep_step_noalloc": (ctypes.c_int, [ctypes.POINTER(sgep_config), _P, _P, ctypes.c_int64,
                                         _P, _P, _P, _P, ctypes.c_int64, _P]),
    "sgep_tc_selftest": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "sgep_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sgep_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libsgep.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of every function declared in include/sgep.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgep_[a-zA-Z_0-9]+)\s*\(", text)))


def check(status: int, where: str) -> int:
    if status < 0:
        detail = lib().sgep_last_error().decode() or lib().sgep_strerror(status).decode()
        raise SgepError(status, where, detail)
    return status


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):          # torch.Tensor
        return x.data_ptr()
    if hasattr(x, "ctypes"):            # numpy.ndarray
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---- thin wrappers with the ABI's names --------------------------------------

def sgep_config_default(**overrides) -> sgep_config:
    cfg = sgep_config()
    check(lib().sgep_config_default(ctypes.byref(cfg)), "sgep_config_default")
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def sgep_init(cfg: sgep_config) -> int:
    h = _P()
    check(lib().sgep_init(ctypes.byref(cfg), ctypes.byref(h)), "sgep_init")
    return h.value


def sgep_destroy(h) -> None:
    check(lib().sgep_destroy(h), "sgep_destroy")


def sgep_step(h, X, Y=None, labels=None, b=None, stream=None, sx=None, sy=None) -> None:
    """sx, sy: per-row scales of FP8 rows (device float arrays), else None."""
    if b is None:
        b = X.shape[0]
    check(lib().sgep_step(h, _ptr(X), _ptr(Y), _ptr(sx), _ptr(sy), _ptr(labels), int(b), _stream(stream)),
          "sgep_step")


def sgep_step_many(h, X, Y, b, nsteps, labels=None, stream=None, sx=None, sy=None) -> None:
    check(lib().sgep_step_many(h, _ptr(X), _ptr(Y), _ptr(sx), _ptr(sy), _ptr(labels), int(b), int(nsteps),
                               _stream(stream)), "sgep_step_many")


def sgep_sync(h, stream=None) -> None:
    check(lib().sgep_sync(h, _stream(stream)), "sgep_sync")


def sgep_get_V(h, out, on_device: bool, stream=None) -> None:
    check(lib().sgep_get_V(h, _ptr(out), int(on_device), _stream(stream)), "sgep_get_V")


def sgep_get_S(h, out, on_device: bool, stream=None) -> None:
    check(lib().sgep_get_S(h, _ptr(out), int(on_device), _stream(stream)), "sgep_get_S")


def sgep_set_V(h, V, on_device: bool, stream=None) -> None:
    check(lib().sgep_set_V(h, _ptr(V), int(on_device), _stream(stream)), "sgep_set_V")


def sgep_set_VS(h, V, S, on_device: bool, stream=None) -> None:
    check(lib().sgep_set_VS(h, _ptr(V), _ptr(S), int(on_device), _stream(stream)), "sgep_set_VS")


def sgep_set_rr_every(h, every, X=None, Y=None, n=0, labels=None, sx=None, sy=None) -> None:
    check(lib().sgep_set_rr_every(h, int(every), _ptr(X), _ptr(Y), _ptr(sx), _ptr(sy), _ptr(labels), int(n)),
          "sgep_set_rr_every")


def sgep_rayleigh_ritz(h, X, Y, n, out=None, labels=None, stream=None, sx=None, sy=None) -> None:
    check(lib().sgep_rayleigh_ritz(h, _ptr(X), _ptr(Y), _ptr(sx), _ptr(sy), _ptr(labels), int(n), _ptr(out),
                                   _stream(stream)), "sgep_rayleigh_ritz")


def sgep_get_eigenvalues(h, X, Y, n, out, labels=None, stream=None, sx=None, sy=None) -> None:
    check(lib().sgep_get_eigenvalues(h, _ptr(X), _ptr(Y), _ptr(sx), _ptr(sy), _ptr(labels), int(n), _ptr(out),
                                     _stream(stream)), "sgep_get_eigenvalues")


def sgep_get_state(h) -> bytes:
    n = ctypes.c_size_t(0)
    check(lib().sgep_get_state(h, None, ctypes.byref(n)), "sgep_get_state")
    buf = ctypes.create_string_buffer(n.value)
    check(lib().sgep_get_state(h, buf, ctypes.byref(n)), "sgep_get_state")
    return buf.raw[: n.value]


def sgep_set_state(h, blob: bytes) -> None:
    check(lib().sgep_set_state(h, blob, len(blob)), "sgep_set_state")


def sgep_step_count(h) -> int:
    return int(lib().sgep_step_count(h))


def sgep_eta_at(h, t: int) -> float:
    return float(lib().sgep_eta_at(h, int(t)))


def sgep_path(h) -> int:
    return check(lib().sgep_path(h), "sgep_path")


def sgep_launch_count(h) -> int:
    return int(lib().sgep_launch_count(h))


def sgep_debug_products(h, AV, BV) -> None:
    check(lib().sgep_debug_products(h, _ptr(AV), _ptr(BV)), "sgep_debug_products")


def sgep_debug_update(h, grad, terms) -> None:
    check(lib().sgep_debug_update(h, _ptr(grad), _ptr(terms)), "sgep_debug_update")


def sgep_step_noalloc(cfg: sgep_config, X, Y, b, V, S, V_out, S_out, t, stream=None) -> None:
    check(lib().sgep_step_noalloc(ctypes.byref(cfg), _ptr(X), _ptr(Y), int(b), _ptr(V), _ptr(S),
                                  _ptr(V_out), _ptr(S_out), int(t), _stream(stream)),
          "sgep_step_noalloc")


def sgep_tc_selftest(mode: int) -> float:
    err = ctypes.c_double(-1.0)
    check(lib().sgep_tc_selftest(int(mode), ctypes.byref(err)), "sgep_tc_selftest")
    return err.value


def sgep_strerror(status: int) -> str:
    return lib().sgep_strerror(status).decode()


def sgep_last_error() -> str:
    return lib().sgep_last_error().decode()


# ---- batching form -----------------------------------------------------------

def _ptr_array(items):
    """Host array of device pointers (None entries become NULL); None if all are None."""
    if items is None:
        return None
    ptrs = [_ptr(x) for x in items]
    if all(p is None for p in ptrs):
        return None
    return (ctypes.c_void_p * len(ptrs))(*ptrs)


def sgep_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    out = ctypes.c_void_p()
    check(lib().sgep_batch_create(arr, len(handles), ctypes.byref(out)), "sgep_batch_create")
    return out


def sgep_batch_destroy(b) -> None:
    check(lib().sgep_batch_destroy(b), "sgep_batch_destroy")


def _rows(rows):
    return (ctypes.c_int64 * len(rows))(*[int(r) for r in rows])


def sgep_batch_step(b, X, Y=None, rows=None, labels=None, sx=None, sy=None, stream=None) -> None:
    check(lib().sgep_batch_step(b, _ptr_array(X), _ptr_array(Y), _ptr_array(sx), _ptr_array(sy),
                                _ptr_array(labels), _rows(rows), _stream(stream)), "sgep_batch_step")


def sgep_batch_sync(b, stream=None) -> None:
    check(lib().sgep_batch_sync(b, _stream(stream)), "sgep_batch_sync")


def sgep_batch_configure(b, mode=-1, blocks_per_sm=0, chunk_cap=0, rows_cap=0, use_graph=-1) -> None:
    check(lib().sgep_batch_configure(b, int(mode), int(blocks_per_sm), int(chunk_cap), int(rows_cap),
                                     int(use_graph)), "sgep_batch_configure")


def sgep_batch_get_config(b):
    out = (ctypes.c_int * 5)()
    check(lib().sgep_batch_get_config(b, out), "sgep_batch_get_config")
    return list(out)


def sgep_batch_autotune(b, X, Y=None, rows=None, labels=None, sx=None, sy=None, reps=3):
    out = (ctypes.c_int * 5)()
    check(lib().sgep_batch_autotune(b, _ptr_array(X), _ptr_array(Y), _ptr_array(sx), _ptr_array(sy),
                                    _ptr_array(labels), _rows(rows), int(reps), out), "sgep_batch_autotune")
    return list(out)


def sgep_batch_launch_count(b) -> int:
    return int(lib().sgep_batch_launch_count(b))


# ---- learned warm start ------------------------------------------------------------

def sgep_sketch(X, Y, dtype, n, d_x, d_y, omega, m, out, stream=None) -> None:
    check(lib().sgep_sketch(_ptr(X), _ptr(Y), int(dtype), int(n), int(d_x), int(d_y), _ptr(omega), int(m),
                            _ptr(out), _stream(stream)), "sgep_sketch")


def sgep_mlp_create(in_dim, out_dim, seed=0):
    out = ctypes.c_void_p()
    check(lib().sgep_mlp_create(int(in_dim), int(out_dim), int(seed), ctypes.byref(out)), "sgep_mlp_create")
    return out


def sgep_mlp_destroy(m) -> None:
    check(lib().sgep_mlp_destroy(m), "sgep_mlp_destroy")


def sgep_mlp_param_count(m) -> int:
    return int(lib().sgep_mlp_param_count(m))


def sgep_mlp_get_params(m, out) -> None:
    check(lib().sgep_mlp_get_params(m, _ptr(out)), "sgep_mlp_get_params")


def sgep_mlp_set_params(m, params) -> None:
    check(lib().sgep_mlp_set_params(m, _ptr(params)), "sgep_mlp_set_params")


def sgep_mlp_forward(m, S, rows, out, stream=None) -> None:
    check(lib().sgep_mlp_forward(m, _ptr(S), int(rows), _ptr(out), _stream(stream)), "sgep_mlp_forward")


def sgep_mlp_loss_grad(m, S, V, seg, n_inst, grad_out=None, stream=None) -> float:
    loss = ctypes.c_double(0.0)
    seg_arr = (ctypes.c_int64 * len(seg))(*[int(x) for x in seg])
    check(lib().sgep_mlp_loss_grad(m, _ptr(S), _ptr(V), seg_arr, int(n_inst), ctypes.byref(loss), _ptr(grad_out),
                                   _stream(stream)), "sgep_mlp_loss_grad")
    return loss.value


def sgep_mlp_adam_step(m, lr, stream=None) -> None:
    check(lib().sgep_mlp_adam_step(m, ctypes.c_float(lr), _stream(stream)), "sgep_mlp_adam_step")
