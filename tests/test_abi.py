"""CPU-side checks of the C ABI: the library builds, loads, exports every entry point the
header declares, its config struct matches ctypes, and host-only logic behaves."""
import ctypes
import os
import subprocess

import pytest

from paper_2206_04993_gb300 import sgep as S


def test_library_exports_every_declared_symbol():
    L = S.lib()
    declared = S.header_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(L, name), name
        assert name in S._SIGS, f"binding lacks {name}"


def test_library_exports_nothing_undeclared():
    out = subprocess.run(["nm", "-D", "--defined-only", S.LIB_PATH], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm not available")
    exported = {ln.split()[-1] for ln in out.stdout.splitlines() if " T sgep_" in ln}
    assert exported == set(S.header_functions())


def test_config_defaults_and_layout():
    cfg = S.sgep_config_default()
    assert cfg.kind == S.SGEP_CCA and cfg.dtype == S.SGEP_F32
    assert cfg.k == 1 and cfg.split_AB == 1 and cfg.max_b == 4096
    assert abs(cfg.rho - 1e-6) < 1e-12 and cfg.schedule == S.SGEP_SCHED_CONST
    assert cfg.machines == 1 and cfg.reserved0 == 0
    # the header's struct: 2 int32, 2 int64, 2 int32, 4 float, 2 int32, 2 int64, float,
    # int32, uint64, int64, int32, 9 int32 (natural alignment)
    assert ctypes.sizeof(S.sgep_config) == 136


def test_strerror_and_null_arguments():
    assert S.sgep_strerror(S.SGEP_OK) == "ok"
    assert S.sgep_strerror(S.SGEP_ENONFINITE) == "non-finite values"
    assert S.sgep_strerror(12345) == "unknown status"
    L = S.lib()
    assert L.sgep_config_default(None) == S.SGEP_EINVAL
    assert L.sgep_init(None, None) == S.SGEP_EINVAL
    assert L.sgep_destroy(None) == S.SGEP_OK
    assert L.sgep_step(None, None, None, None, None, None, 4, None) == S.SGEP_EINVAL
    assert L.sgep_step_count(None) == -1


@pytest.mark.parametrize("field,value", [
    ("k", 0), ("k", 65), ("d_x", 0), ("rho", 0.0), ("kind", 9), ("dtype", 7),
    ("max_b", 1), ("schedule", 5), ("path", 9),
])
def test_init_rejects_bad_config_before_touching_the_gpu(field, value):
    cfg = S.sgep_config_default(d_x=8, d_y=8, k=2)
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    rc = S.lib().sgep_init(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == S.SGEP_EINVAL and h.value is None
    assert S.sgep_last_error() != ""


def test_init_rejects_shape_and_schedule_mismatch():
    L = S.lib()
    h = ctypes.c_void_p()
    cfg = S.sgep_config_default(kind=S.SGEP_PCA, d_x=8, d_y=3, k=2)
    assert L.sgep_init(ctypes.byref(cfg), ctypes.byref(h)) == S.SGEP_EINVAL
    cfg = S.sgep_config_default(d_x=2, d_y=1, k=4)
    assert L.sgep_init(ctypes.byref(cfg), ctypes.byref(h)) == S.SGEP_EINVAL
    cfg = S.sgep_config_default(d_x=8, d_y=8, k=2, schedule=2, t_c=10, T=5, eta_T=0.01)
    assert L.sgep_init(ctypes.byref(cfg), ctypes.byref(h)) == S.SGEP_EINVAL
    cfg = S.sgep_config_default(kind=S.SGEP_LDA, d_x=8, d_y=0, k=2)  # n_classes missing
    assert L.sgep_init(ctypes.byref(cfg), ctypes.byref(h)) == S.SGEP_EINVAL
    cfg = S.sgep_config_default(kind=S.SGEP_LDA, d_x=8, d_y=2, k=2, n_classes=3)  # LDA has one view
    assert L.sgep_init(ctypes.byref(cfg), ctypes.byref(h)) == S.SGEP_EINVAL
    cfg = S.sgep_config_default(kind=S.SGEP_LDA, d_x=8, d_y=0, k=2, n_classes=33)
    assert L.sgep_init(ctypes.byref(cfg), ctypes.byref(h)) == S.SGEP_EINVAL


@pytest.mark.parametrize("fields,why", [
    ({"optimizer": 7}, "optimizer"),
    ({"optimizer": S.SGEP_OPT_ADAM, "adam_b1": 1.0}, "Adam"),
    ({"optimizer": S.SGEP_OPT_ADAM, "adam_b2": -0.1}, "Adam"),
    ({"optimizer": S.SGEP_OPT_ADAM, "adam_eps": float("inf")}, "Adam"),
    ({"variant": 5}, "variant"),
    ({"variant": S.SGEP_ALG3, "nu": float("inf")}, "nu"),
    ({"center": 2}, "center"),
])
def test_init_rejects_bad_variant_config_before_touching_the_gpu(fields, why):
    """Adam (App. H.2.2), Alg. 3 (App. E.2) and running-mean centring settings are checked
    before any device work, each with its own message."""
    cfg = S.sgep_config_default(d_x=8, d_y=8, k=2)
    for name, value in fields.items():
        setattr(cfg, name, value)
    h = ctypes.c_void_p()
    assert S.lib().sgep_init(ctypes.byref(cfg), ctypes.byref(h)) == S.SGEP_EINVAL and h.value is None
    assert why in S.sgep_last_error(), S.sgep_last_error()


def test_init_rejects_variant_and_kind_combinations():
    L = S.lib()
    h = ctypes.c_void_p()
    cfg = S.sgep_config_default(d_x=8, d_y=8, k=2, variant=S.SGEP_ALG3)
    cfg.nu = cfg.rho  # Alg. 3 interpolates between rho and nu > rho
    assert L.sgep_init(ctypes.byref(cfg), ctypes.byref(h)) == S.SGEP_EINVAL
    cfg = S.sgep_config_default(kind=S.SGEP_ICA, d_x=8, d_y=4, k=2)  # ICA has one view
    assert L.sgep_init(ctypes.byref(cfg), ctypes.byref(h)) == S.SGEP_EINVAL
    cfg = S.sgep_config_default(kind=S.SGEP_LDA, d_x=8, d_y=0, k=2, n_classes=3, center=1)
    assert L.sgep_init(ctypes.byref(cfg), ctypes.byref(h)) == S.SGEP_EINVAL  # LDA centres by class


def test_init_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = S.sgep_config_default(d_x=8, d_y=8, k=2)
    h = ctypes.c_void_p()
    rc = S.lib().sgep_init(ctypes.byref(cfg), ctypes.byref(h))
    assert rc in (S.SGEP_ECUDA, S.SGEP_ENOMEM) and h.value is None


def test_product_path_does_not_reach_the_oracle():
    pkg = os.path.dirname(S.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(root, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
