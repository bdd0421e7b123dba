"""Benchmark of the gamma-EigenGame step (Alg. 2) on GB300.

Default workload: activation-like CCA, d_x = d_y = 16384 (d = 32768), k = 32 players,
minibatch b = 4096 rows in BF16 (268 MB per minibatch), power-law noise spectrum with 64
planted shared directions. A pool of 262,144 rows (64 minibatches, 17.2 GB) is generated on
the device before timing; timed steps stream consecutive minibatches through it (one launch
runs up to 64 of them), so the inputs exceed L2 and every step reads fresh rows from HBM. The other workloads (the
1024-dim FP32 CCA with its time-to-1e-3 runs, the FP32 form of the large problem, the
batching form, the learned warm start) are reported under `forms`.

One JSON line is printed (rank 0). `value` is samples/s of the whole job with inputs
resident in HBM; `e2e` is the same metric through the C ABI with the minibatch copied
from pinned host memory and V read back every step; `roofline` relates the step's
algorithmic bytes to the measured HBM peak; `cpu_baseline` is the FP64 oracle timed on
this host's cores on a bounded sample.

  python bench.py [--gpus N --steps K --warmup W] [--workload NAME] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "samples/s and time-to-1e-3 gen.-subspace error: plain FP32 vs BF16/batched/warm"

WORKLOADS = {
    # name: (synth config function, dtype, pool rows)
    "cca_d1024_k16_b1024_f32": ("config_c2", "f32", 1_000_000),
    "cca_d64_k4_b256_f32": ("config_c1", "f32", 10_000),
    # activation-like CCA, d_x = d_y = 16384, k = 32, b = 4096, BF16 rows (64 minibatches = 17.2 GB)
    "cca_d32768_k32_b4096_bf16": ("config_c3", "bf16", 262_144),
    "cca_d32768_k32_b4096_f32": ("config_c3", "f32", 16_384),
}
DEFAULT_WORKLOAD = "cca_d32768_k32_b4096_bf16"
TTE_WORKLOAD = "cca_d1024_k16_b1024_f32"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--path", type=int, default=0, help="0 auto, 1 generic, 2 cluster, 3 tc")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--pool-rows", type=int, default=0, help="override the resident row pool")
    p.add_argument("--no-tte", action="store_true", help="skip the time-to-1e-3 measurements")
    p.add_argument("--no-forms", action="store_true", help="skip the BF16 tensor-core and batching workloads")
    p.add_argument("--tte-max-steps", type=int, default=80_000)
    return p.parse_args()


# DRAM bytes (read + write) per step of the dominant kernel from one ncu capture of the
# current kernel (profiles/); an entry is removed whenever the kernel changes until it is
# captured again.
TRAFFIC_BYTES = {
    # k_tc_stream: (645.3 MB read + 20.1 MB written) in one launch of 2 steps, from the ncu
    # capture summarised under profiles/
    "cca_d32768_k32_b4096_bf16": 327_665_664,
}


def world_max(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank timing over all ranks (one all-reduce; identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region

def gpu_selector(dev) -> str:
    """The nvidia-smi `-i` argument of the GPU behind torch device `dev`: its UUID (CUDA
    ordinals are relative to CUDA_VISIBLE_DEVICES, nvidia-smi indices are not)."""
    import torch
    idx = torch.device(dev).index or 0
    try:
        u = str(torch.cuda.get_device_properties(idx).uuid)
        if u:
            return u if u.startswith(("GPU-", "MIG-")) else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if idx < len(ids):
            return ids[idx]
    return str(idx)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.idx = gpu_selector(dev)
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "gpu": self.idx}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# data

def make_pool(cfg, rows, dtype, device, seed=0):
    """Rows of the planted CCA model generated on the device (torch RNG)."""
    import torch
    model = cfg["model"]
    g = torch.Generator(device=device)
    g.manual_seed(1000 + seed)
    Wx = torch.from_numpy(model.Wx).float().to(device)
    Wy = torch.from_numpy(model.Wy).float().to(device)
    r = Wx.shape[1]
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    X = torch.empty(rows, model.d_x, device=device, dtype=tdt)
    Y = torch.empty(rows, model.d_y, device=device, dtype=tdt)
    if hasattr(model, "sigma"):
        sx = sy = None
    else:
        sx = torch.from_numpy(np.sqrt(model.Dx)).float().to(device)
        sy = torch.from_numpy(np.sqrt(model.Dy)).float().to(device)
    chunk = max(1, min(1 << 17, (1 << 28) // max(model.d_x, 1)))
    for r0 in range(0, rows, chunk):
        n = min(chunk, rows - r0)
        z = torch.randn(n, r, device=device, generator=g)
        ex = torch.randn(n, model.d_x, device=device, generator=g)
        ey = torch.randn(n, model.d_y, device=device, generator=g)
        if sx is None:
            X[r0:r0 + n] = (z @ Wx.T + model.sigma * ex).to(tdt)
            Y[r0:r0 + n] = (z @ Wy.T + model.sigma * ey).to(tdt)
        else:
            X[r0:r0 + n] = (z @ Wx.T + ex * sx).to(tdt)
            Y[r0:r0 + n] = (z @ Wy.T + ey * sy).to(tdt)
    return X, Y


# ---------------------------------------------------------------------------
# time-to-error: ground truth of the resident row pool, as the paper takes it (scipy's dense
# symmetric generalized solver on the finite-sample covariances, Sec. 5)

def pool_truth(X, Y, k, chunk=65536):
    import scipy.linalg as sla
    n, dx = X.shape
    dy = Y.shape[1]
    Cxx = np.zeros((dx, dx))
    Cyy = np.zeros((dy, dy))
    Cxy = np.zeros((dx, dy))
    for r0 in range(0, n, chunk):
        xc = X[r0:r0 + chunk].float().cpu().numpy().astype(np.float64)
        yc = Y[r0:r0 + chunk].float().cpu().numpy().astype(np.float64)
        Cxx += xc.T @ xc
        Cyy += yc.T @ yc
        Cxy += xc.T @ yc
    d = dx + dy
    A = np.zeros((d, d))
    B = np.zeros((d, d))
    A[:dx, dx:] = Cxy / n
    A[dx:, :dx] = Cxy.T / n
    B[:dx, :dx] = Cxx / n
    B[dx:, dx:] = Cyy / n
    w, U = sla.eigh(A, B, subset_by_index=[d - k, d - 1])
    return U[:, ::-1].copy(), B, w[::-1].copy()


def gen_subspace_error(Vt, Vh, B):
    """1 - tr(U* P)/k of App. A.1 in Gram form."""
    BVt, BVh = B @ Vt, B @ Vh
    Gth = Vt.T @ BVh
    tr = np.trace(np.linalg.solve(Vt.T @ BVt, Gth) @ np.linalg.solve(Vh.T @ BVh, Gth.T))
    return float(1.0 - tr / Vt.shape[1])


def lowrank_cca_truth(model, k):
    """Population top-k solution of the activation-like CCA model (Cxx = Dx + Wx Wx^T,
    Cyy = Dy + Wy Wy^T, Cxy = Wx Wy^T, Dx, Dy diagonal, rank-m W) without a d x d matrix.
    With a = Cxx^-1 Wx alpha and b = Cyy^-1 Wy beta the pencil reduces to Gy Gx alpha =
    lambda^2 alpha, beta = Gx alpha / lambda, where Gx = Wx^T Cxx^-1 Wx (m x m) and
    Cxx^-1 Wx = Dx^-1 Wx (I + Wx^T Dx^-1 Wx)^-1 (Woodbury). Returns (V*, lambda, B-apply)."""
    import scipy.linalg as sla

    def cinv_w(D, W):
        DW = W / D[:, None]
        return DW @ np.linalg.inv(np.eye(W.shape[1]) + W.T @ DW)

    Cx, Cy = cinv_w(model.Dx, model.Wx), cinv_w(model.Dy, model.Wy)
    Gx, Gy = model.Wx.T @ Cx, model.Wy.T @ Cy
    Gx, Gy = 0.5 * (Gx + Gx.T), 0.5 * (Gy + Gy.T)
    wx, Ux = sla.eigh(Gx)
    Gh = (Ux * np.sqrt(wx)) @ Ux.T
    Gih = (Ux / np.sqrt(wx)) @ Ux.T
    lam2, U = sla.eigh(Gh @ Gy @ Gh)
    order = np.argsort(lam2)[::-1][:k]
    lam = np.sqrt(np.maximum(lam2[order], 0.0))
    alpha = Gih @ U[:, order]
    beta = Gx @ alpha / lam[None, :]
    V = np.concatenate([Cx @ alpha, Cy @ beta])
    V /= np.linalg.norm(V, axis=0, keepdims=True)
    dx = model.Dx.size

    def Bmv(U_):
        ux, uy = U_[:dx], U_[dx:]
        return np.concatenate([model.Dx[:, None] * ux + model.Wx @ (model.Wx.T @ ux),
                               model.Dy[:, None] * uy + model.Wy @ (model.Wy.T @ uy)])
    return V, lam, Bmv


def gen_subspace_error_op(Vt, Vh, Bmv):
    """gen_subspace_error with B applied through an operator (no d x d matrix)."""
    BVt, BVh = Bmv(Vt), Bmv(Vh)
    Gth = Vt.T @ BVh
    tr = np.trace(np.linalg.solve(Vt.T @ BVt, Gth) @ np.linalg.solve(Vh.T @ BVh, Gth.T))
    return float(1.0 - tr / Vt.shape[1])


def time_to_error(make_solver, X, Y, b, truth, target=1e-3, every=500, max_steps=80_000, seed=123):
    """Steps and device seconds from the cold start v_i ~ N(0, I) (normalised) until the
    generalized subspace error against `truth` is at most `target`; the error is evaluated
    every `every` steps outside the timed region."""
    import torch
    Vs, B, _ = truth
    d, k = Vs.shape
    solver = make_solver()
    solver.set_V(synth.random_unit_columns(d, k, seed=seed).astype(np.float32))
    nb = X.shape[0] // b
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pos, ms, err = 0, 0.0, 1.0
    curve = []
    # Epochs over the pool; odd epochs shift the minibatch grid by b/2 rows so that every row
    # estimates A in one epoch and B in the next (the split of Alg. 2's independent batches).
    per = [nb, nb - 1]
    while pos < max_steps:
        n = min(every, max_steps - pos)
        e0.record()
        left, s0 = n, pos
        while left > 0:
            ep, j = divmod(s0, nb + nb - 1)
            odd = j >= nb
            j = j - nb if odd else j
            m = min(left, per[odd] - j)
            r0 = j * b + (b // 2 if odd else 0)
            solver.step_many(X[r0:r0 + m * b], Y[r0:r0 + m * b], b, m)
            s0 += m
            left -= m
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        pos += n
        err = gen_subspace_error(Vs, solver.V().astype(np.float64), B)
        curve.append((pos, round(err, 6)))
        if err <= target:
            break
    solver.close()
    return {"target": target, "reached": err <= target, "steps": pos, "seconds": ms / 1e3,
            "samples": pos * b, "final_error": err, "curve_every": every,
            "curve": curve[:: max(1, len(curve) // 12)]}


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle on host cores

def oracle_rate(cfg, seconds: float):
    """Samples/s of the oracle's Alg. 2 step (FP64, numpy, streamed operators) on
    minibatches of the workload, over about `seconds` of work (at least two steps)."""
    from oracle import eg
    model = cfg["model"]
    b, k = cfg["b"], cfg["k"]
    d = model.d_x + model.d_y
    V = synth.random_unit_columns(d, k, seed=0)
    S = V.copy()
    nbat = 4 if b * d <= 1 << 24 else 2  # two FP64 minibatches (2.1 GB) at the 32768-dim size
    batches = [synth.draw_rows(model, b, batch=i) for i in range(nbat)]
    steps = 0
    t0 = time.perf_counter()
    while True:
        X, Y = batches[steps % nbat]
        V, S = eg.eg_step(V, S, *eg.cca_ops(X, Y), cfg["eta0"], cfg["gamma0"], cfg["rho"])
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds and steps >= 2:
            break
    return steps * b / el, steps, el


def line_config(workload: str, pool_rows: int, world: int) -> dict:
    """The `config` block of the JSON line; both arms print the same one."""
    cfg = getattr(synth, WORKLOADS[workload][0])()
    model = cfg["model"]
    return {"workload": workload, "d_x": model.d_x, "d_y": model.d_y, "k": cfg["k"], "b": cfg["b"],
            "dtype": WORKLOADS[workload][1], "pool_rows": pool_rows,
            "l2": "inputs larger than L2 (pool streamed)", "parallelism": f"replicas{world}"}


def fma_roofline(b, d, k, ms, n_sms, sm_mhz, sm_max_mhz=None, split=True):
    """FP32 FMA-rate roofline of the SIMT contractions: the projection does k FMAs per
    element, the back-projection k with split A/B batches (every row feeds one estimate) or 2k
    without; the peak is n_sms x 128 FP32 FMA per clock at the SM clock sampled during the
    timed region (the rated maximum is reported beside it)."""
    fma = b * d * k * (2 if split else 3)
    peak = n_sms * 128 * sm_mhz * 1e6 / 1e12
    achieved = fma / (ms / 1e3) / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFMA/s", "frac": achieved / peak,
           "fma_per_step": fma, "kernel": "generic projection + back-projection (whole step)",
           "peak_source": f"{n_sms} SMs x 128 FP32 FMA/clock x {sm_mhz:.0f} MHz (median sampled SM clock)"}
    if sm_max_mhz:
        pmax = n_sms * 128 * sm_max_mhz * 1e6 / 1e12
        out["at_rated_max_clock"] = {"peak": pmax, "frac": achieved / pmax, "sm_mhz": sm_max_mhz}
    return out


def measure_throughput(workload, steps, warmup, dev, rank=0, path=0):
    """Samples/s and roofline of one workload with its rows resident in HBM."""
    import torch
    from paper_2206_04993_gb300 import Solver, sgep
    name, dtype, pool_rows = WORKLOADS[workload]
    cfg = getattr(synth, name)(seed=rank)
    model = cfg["model"]
    b, k = cfg["b"], cfg["k"]
    dx, dy = model.d_x, model.d_y
    d = dx + dy
    esz = 2 if dtype == "bf16" else 4
    X, Y = make_pool(cfg, pool_rows, dtype, dev, seed=rank)
    nb = pool_rows // b
    solver = Solver(kind=sgep.SGEP_CCA, d_x=dx, d_y=dy, k=k,
                    dtype=sgep.SGEP_BF16 if dtype == "bf16" else sgep.SGEP_F32,
                    eta0=cfg["eta0"], gamma0=cfg["gamma0"], rho=cfg["rho"], max_b=b, path=path, seed=rank)
    def run(start, count):  # consecutive minibatches of the pool, as few sgep_step_many calls as it allows
        i = 0
        while i < count:
            j = (start + i) % nb
            n = min(count - i, nb - j)
            solver.step_many(X[j * b:(j + n) * b], Y[j * b:(j + n) * b], b, n)
            i += n

    run(0, warmup)
    solver.sync()
    torch.cuda.synchronize()
    l0 = solver.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        e0.record()
        run(warmup, steps)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    peak, peak_kind = measured_peaks()
    alg = b * d * esz + 16 * d * k
    out = {"value": b / (ms / 1e3), "unit": "samples/s", "ms_per_step": ms, "dtype": dtype,
           "path": solver.path, "gpu_launches": solver.launches - l0, "steps": steps, "warmup": warmup,
           "config": {"d_x": dx, "d_y": dy, "k": k, "b": b, "pool_rows": pool_rows},
           "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": None,
                        "kernel": "whole step", "peak_source": peak_kind, "alg_bytes_per_launch": alg},
           "clocks": clk.summary()}
    if dtype == "f32" and solver.path == sgep.SGEP_PATH_GENERIC:  # SIMT contractions: FMA-bound
        try:
            mhz = out["clocks"].get("sm_mhz") or out["clocks"].get("sm_max_mhz")
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            if mhz:
                out["fma_roofline"] = fma_roofline(b, d, k, ms, sms, float(mhz), out["clocks"].get("sm_max_mhz"))
        except Exception:  # an extra figure: never costs the measurement
            pass
    solver.close()
    del X, Y
    torch.cuda.empty_cache()
    return out


def measure_batch(dtype, steps, warmup, dev, seed=0, n_instances=64):
    """Batching workload: 64 uneven instances (half CCA, half LDA), b = 512 each, advanced by
    one batched launch per step (configuration from the autotuner), against the same
    instances stepped one handle at a time. Rows: two resident minibatches per instance."""
    import torch
    from paper_2206_04993_gb300 import Batch, Solver, sgep
    insts = synth.config_c4(seed=seed, n_instances=n_instances)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    g = torch.Generator(device=dev)
    g.manual_seed(seed + 17)
    rows = []  # per instance: list of (X, Y, labels) for two minibatches
    for it in insts:
        b = it["b"]
        m = it["model"]
        mbs = []
        for _ in range(2):
            if it["kind"] == "cca":
                Wx = torch.tensor(m.Qx * m.s, dtype=torch.float32, device=dev)
                Wy = torch.tensor(m.Qy * m.s, dtype=torch.float32, device=dev)
                z = torch.randn(b, m.s.size, device=dev, generator=g)
                X = z @ Wx.T + m.sigma * torch.randn(b, it["d_x"], device=dev, generator=g)
                Y = z @ Wy.T + m.sigma * torch.randn(b, it["d_y"], device=dev, generator=g)
                mbs.append((X.to(tdt).contiguous(), Y.to(tdt).contiguous(), None))
            else:
                C = it["n_classes"]
                lab = torch.randint(0, C, (b,), device=dev, generator=g, dtype=torch.int32)
                means = torch.tensor(m["means"], dtype=torch.float32, device=dev)
                sc = torch.tensor(m["scales"], dtype=torch.float32, device=dev)
                X = means[lab.long()] + torch.randn(b, it["d_x"], device=dev, generator=g) * sc
                mbs.append((X.to(tdt).contiguous(), None, lab))
        rows.append(mbs)
    dt = sgep.SGEP_BF16 if dtype == "bf16" else sgep.SGEP_F32

    def make():
        out = []
        for i, it in enumerate(insts):
            out.append(Solver(kind=sgep.SGEP_CCA if it["kind"] == "cca" else sgep.SGEP_LDA, d_x=it["d_x"],
                              d_y=it["d_y"], k=it["k"], n_classes=it.get("n_classes", 0), max_b=it["b"], dtype=dt,
                              path=sgep.SGEP_PATH_GENERIC, eta0=0.05, gamma0=0.3, seed=i))
        return out

    def args_of(j):
        return ([r[j][0] for r in rows], [r[j][1] for r in rows], [it["b"] for it in insts],
                [r[j][2] for r in rows])

    samples = sum(it["b"] for it in insts)
    alg = sum(it["b"] * (it["d_x"] + it["d_y"]) * (2 if dtype == "bf16" else 4) for it in insts)
    solvers = make()
    out = {"unit": "samples/s", "dtype": dtype, "instances": len(insts),
           "config": {"kinds": "even CCA (d 64..4096, d_x = d_y), odd LDA (10 classes)", "k": "4..32 (LDA <= 9)",
                      "b": 512, "d_total": int(sum(it["d_x"] + it["d_y"] for it in insts))}}
    with Batch(solvers) as bt:
        X0, Y0, R0, L0 = args_of(0)
        bt.configure(use_graph=1)
        out["autotuned"] = dict(zip(["mode", "blocks_per_sm", "chunk_cap", "rows_cap", "use_graph"],
                                    bt.autotune(X0, Y0, R0, labels=L0, reps=3)))
        for i in range(warmup):
            Xs, Ys, Rs, Ls = args_of(i % 2)
            bt.step(Xs, Ys, Rs, labels=Ls)
        bt.sync()
        torch.cuda.synchronize()
        l0 = bt.launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(steps):
            Xs, Ys, Rs, Ls = args_of(i % 2)
            bt.step(Xs, Ys, Rs, labels=Ls)
        e1.record()
        torch.cuda.synchronize()
        bt.sync()
        ms = e0.elapsed_time(e1) / steps
        out.update({"value": samples / (ms / 1e3), "ms_per_step": ms,
                    "gpu_launches_per_step": (bt.launches() - l0) / steps,
                    "algorithmic_GBps": alg / (ms / 1e3) / 1e9})
    # the same instances stepped one handle at a time (generic path, one stream)
    for i in range(warmup):
        Xs, Ys, Rs, Ls = args_of(i % 2)
        for s, x, y, r, lb in zip(solvers, Xs, Ys, Rs, Ls):
            s.step(x, y, r, labels=lb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    seq_steps = max(3, steps // 4)
    e0.record()
    for i in range(seq_steps):
        Xs, Ys, Rs, Ls = args_of(i % 2)
        for s, x, y, r, lb in zip(solvers, Xs, Ys, Rs, Ls):
            s.step(x, y, r, labels=lb)
    e1.record()
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1) / seq_steps
    out["one_by_one"] = {"value": samples / (ms_seq / 1e3), "ms_per_step": ms_seq, "steps": seq_steps}
    out["speedup_vs_one_by_one"] = ms_seq / ms
    for s in solvers:
        s.close()
    del rows
    torch.cuda.empty_cache()
    return out


def measure_warm(dev, seed=0, n_train=128, n_eval=16, max_steps=8000, check_every=200, target=1e-3):
    """Learned warm start on a planted CCA family (d_x = d_y = 64, k = 4, 8 latent directions,
    mixing matrices a smooth function of theta in [-1, 1]^8; reduced from the full-size family,
    d_x = d_y = 1024, k = 16, 4096 instances, to fit the bench's time budget). The network is
    trained on the plain solver's solutions of n_train instances; on n_eval held-out instances
    the plain iteration runs from the network's V0 (warm) and from random V0 (cold) with the
    same schedule; truth = the exact solution of each instance's resident row pool."""
    import torch
    from paper_2206_04993_gb300 import Batch, Solver, WarmStart, sgep
    fam = synth.config_c5(seed=seed + 1, d_x=64, k=4, latent=8, spread=0.3)
    d_x, k, b, nmb = 64, 4, 512, 32
    d = 2 * d_x
    g = torch.Generator(device=dev)
    g.manual_seed(seed + 29)
    om = torch.tensor(fam["omega"], dtype=torch.float32, device=dev)

    def pool(model):
        Wx = torch.tensor(model.Qx * model.s, dtype=torch.float32, device=dev)
        Wy = torch.tensor(model.Qy * model.s, dtype=torch.float32, device=dev)
        z = torch.randn(nmb * b, model.s.size, device=dev, generator=g)
        X = z @ Wx.T + 0.5 * torch.randn(nmb * b, d_x, device=dev, generator=g)
        Y = z @ Wy.T + 0.5 * torch.randn(nmb * b, d_x, device=dev, generator=g)
        # b/2 wrap-around rows so that odd epochs can shift the minibatch grid by b/2
        return torch.cat([X, X[:b // 2]]).contiguous(), torch.cat([Y, Y[:b // 2]]).contiguous()

    def solvers(n, V0=None):
        # hold then harmonic: eta_t = 0.2 (100 + 20) / (t + 20) after t = 100 (the 64-dim workload's schedule)
        ss = [Solver(kind=sgep.SGEP_CCA, d_x=d_x, d_y=d_x, k=k, max_b=b, path=sgep.SGEP_PATH_GENERIC, eta0=0.2,
                     gamma0=0.3, rho=1e-6, schedule=sgep.SGEP_SCHED_HOLD_HARMONIC, t_c=100, T=max_steps,
                     eta_T=0.2 * 120.0 / (max_steps + 20.0), seed=500 + i) for i in range(n)]
        if V0 is not None:
            for s_, v in zip(ss, V0):
                s_.set_V(v)
        return ss

    def run(bt, pools, t0, count):
        # odd epochs shift the grid by b/2 so that every row estimates A and B equally often
        for t in range(t0, t0 + count):
            o = (t // nmb) % 2 * (b // 2) + (t % nmb) * b
            bt.step([X[o:o + b] for X, _ in pools], [Y[o:o + b] for _, Y in pools], [b] * len(pools))

    train = [fam["model"](t) for t in fam["thetas"](n_train, 0)]
    held = [fam["model"](t) for t in fam["thetas"](n_eval, 1)]
    tp = [pool(m) for m in train]
    ts = solvers(n_train)
    with Batch(ts) as bt:
        run(bt, tp, 0, 1000)
        bt.sync()
    targets = torch.tensor(np.concatenate([s_.V() for s_ in ts]), device=dev)
    for s_ in ts:
        s_.close()
    t_start = time.time()
    sk_train = torch.cat([WarmStart.sketch(X[:2048], Y[:2048], om) for X, Y in tp])
    del tp
    ws = WarmStart(m=16, k=k, seed=seed + 3)
    seg = [i * d for i in range(n_train + 1)]
    first = ws.loss_grad(sk_train, targets, seg)
    for _ in range(300):
        last = ws.loss_grad(sk_train, targets, seg)
        ws.adam_step(3e-3)
    train_s = time.time() - t_start
    hp = [pool(m) for m in held]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ws.forward(WarmStart.sketch(hp[0][0][:2048], hp[0][1][:2048], om))  # warm-up (first-call set-up)
    torch.cuda.synchronize()
    t_inf = time.time()
    e0.record()
    outs = [ws.forward(WarmStart.sketch(X[:2048], Y[:2048], om)) for X, Y in hp]  # sketch + network
    e1.record()
    torch.cuda.synchronize()
    infer_ms = (time.time() - t_inf) * 1e3 / n_eval
    infer_dev_ms = e0.elapsed_time(e1) / n_eval
    V0 = []
    for o in outs:  # unit columns (the players' sphere)
        v = o.cpu().numpy().astype(np.float64)
        V0.append((v / np.linalg.norm(v, axis=0, keepdims=True)).astype(np.float32))
    truths = []
    for X, Y in hp:  # exact top-k solution of the pool (scipy, FP64), the unique rows only
        Z = torch.cat([X[:nmb * b], Y[:nmb * b]], dim=1).double()
        C = (Z.T @ Z / Z.shape[0]).cpu().numpy()
        A = np.zeros_like(C)
        A[:d_x, d_x:] = C[:d_x, d_x:]
        A[d_x:, :d_x] = C[d_x:, :d_x]
        B = np.zeros_like(C)
        B[:d_x, :d_x] = C[:d_x, :d_x]
        B[d_x:, d_x:] = C[d_x:, d_x:]
        import scipy.linalg as sla
        w, U = sla.eigh(A, B)
        truths.append((U[:, ::-1][:, :k], B))
    out = {"scale": "reduced: d_x = d_y = 64, k = 4, latent 8, 128 training / 16 held-out instances",
           "train_loss": [first, last], "train_seconds_host": train_s,
           "warm_start_inference_ms_per_instance": {"wall": infer_ms, "device": infer_dev_ms},
           "target": target, "truth": "exact solution of each held-out instance's resident row pool"}
    # Both starts run the same number of batched steps (max_steps); an instance's steps to the
    # target are read off its error every check_every steps, and the device time to the target
    # is those steps times the measured time per batched step divided by the batch size (the
    # batch runs all instances at once), so neither start is charged for the other instances.
    for name, init in (("cold", None), ("warm", V0)):
        ss = solvers(n_eval, init)
        reached = [None] * n_eval
        err0 = [gen_subspace_error(Vt, s_.V().astype(np.float64), B) for s_, (Vt, B) in zip(ss, truths)]
        dev_ms = 0.0
        curve = []
        err_at = {}
        with Batch(ss) as bt:
            t = 0
            while t < max_steps:
                e0.record()
                run(bt, hp, t, check_every)
                e1.record()
                torch.cuda.synchronize()
                dev_ms += e0.elapsed_time(e1)
                t += check_every
                errs = []
                for i, (s_, (Vt, B)) in enumerate(zip(ss, truths)):
                    e = gen_subspace_error(Vt, s_.V().astype(np.float64), B)
                    errs.append(e)
                    if reached[i] is None and e <= target:
                        reached[i] = t
                if t in (200, 1000, max_steps):
                    err_at[t] = float(np.median(errs))
                if t % (5 * check_every) == 0:
                    curve.append([t, round(float(np.median(errs)), 6)])
            bt.sync()
        ms_per_step = dev_ms / t
        steps = [r for r in reached if r is not None]
        med = float(np.median([r if r is not None else np.inf for r in reached]))
        out[name] = {"initial_error_median": float(np.median(err0)), "reached": len(steps), "of": n_eval,
                     "median_steps_to_target": med if np.isfinite(med) else None,
                     "median_device_seconds_to_target_per_instance":
                         med * ms_per_step / 1e3 / n_eval if np.isfinite(med) else None,
                     "median_error_at_steps": err_at, "steps_run": t,
                     "batched_step_ms": ms_per_step, "median_error_curve": curve}
        for s_ in ss:
            s_.close()
    ws.close()
    torch.cuda.empty_cache()
    return out


def measure_batch_tte(dev, seed=0, n=16, b=512, nmb=32, max_steps=60_000, every=1000, target=1e-3):
    """Time to 1e-3 of the batching form against the same instances stepped alone. Instances: the
    CCA half of the batching workload's generator (planted CCA, 16 latent directions with
    correlations 0.9..0.3, noise 0.5) restricted to d_x = d_y <= 512 and k <= 12, so that the exact
    FP64 solution of every instance's resident pool (nmb minibatches of b rows) is cheap. Every
    start runs the same harmonic schedule on the same pool sequence (odd epochs shift the
    minibatch grid by b / 2 so that every row estimates A and B equally often). Device time of
    the steps only; the errors are evaluated every `every` steps outside it."""
    import torch
    from paper_2206_04993_gb300 import Batch, Solver, sgep
    rng = np.random.default_rng(seed + 41)
    insts = []
    for i in range(n):
        dx = int(rng.integers(32, 513))
        k = int(rng.integers(4, 13))
        insts.append((dx, k, synth.planted_cca(dx, dx, np.linspace(0.9, 0.3, 16), sigma=0.5, seed=9000 + i)))
    pools, truths = [], []
    for i, (dx, k, m) in enumerate(insts):
        X, Y = make_pool({"model": m}, nmb * b, "f32", dev, seed=7000 + i)
        truths.append(pool_truth(X, Y, k))
        pools.append((torch.cat([X, X[:b // 2]]).contiguous(), torch.cat([Y, Y[:b // 2]]).contiguous()))
    sched = dict(eta0=0.2, gamma0=0.3, rho=1e-6, schedule=sgep.SGEP_SCHED_HOLD_HARMONIC, t_c=1, T=20_000,
                 eta_T=0.2 * 401.0 / 20_400.0)

    def offset(t):  # first row of step t's minibatch in the pool
        return (t // nmb) % 2 * (b // 2) + (t % nmb) * b

    def mk(i, path):
        dx, k, _ = insts[i]
        s_ = Solver(kind=sgep.SGEP_CCA, d_x=dx, d_y=dx, k=k, max_b=b, path=path, seed=100 + i, **sched)
        s_.set_V(synth.random_unit_columns(2 * dx, k, seed=300 + i).astype(np.float32))
        return s_

    def err(i, s_):
        Vs, B, _ = truths[i]
        return gen_subspace_error(Vs, s_.V().astype(np.float64), B)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"instances": n, "b": b, "pool_rows": nmb * b, "target": target,
           "config": "CCA, d_x = d_y uniform in 32..512, k uniform in 4..12, 16 planted directions (0.9..0.3)",
           "truth": "scipy eigh of each pool's FP64 covariances"}
    # the batch: every instance advances by one step per batched step until all reach the target
    ss = [mk(i, sgep.SGEP_PATH_GENERIC) for i in range(n)]
    reached = [None] * n
    ms, t = 0.0, 0
    with Batch(ss) as bt:
        bt.configure(use_graph=1)
        # the launch mode and partition the autotuner picks (it restores every instance's state)
        out["autotuned"] = dict(zip(["mode", "blocks_per_sm", "chunk_cap", "rows_cap", "use_graph"],
                                    bt.autotune([X[:b] for X, _ in pools], [Y[:b] for _, Y in pools], [b] * n,
                                                reps=3)))
        while t < max_steps and any(r is None for r in reached):
            e0.record()
            for u in range(t, t + every):
                o = offset(u)
                bt.step([X[o:o + b] for X, _ in pools], [Y[o:o + b] for _, Y in pools], [b] * n)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            t += every
            for i in range(n):
                if reached[i] is None and err(i, ss[i]) <= target:
                    reached[i] = t
        bt.sync()
    final = [round(err(i, ss[i]), 6) for i in range(n)]
    for s_ in ss:
        s_.close()
    out["batched"] = {"reached": sum(r is not None for r in reached), "steps_to_all": t,
                      "device_seconds_to_all": ms / 1e3, "ms_per_batched_step": ms / t,
                      "steps_per_instance": reached, "final_error_per_instance": final,
                      "d_x_per_instance": [it[0] for it in insts], "k_per_instance": [it[1] for it in insts]}
    # one instance at a time, the same steps: generic handles (as in the batch), and the path the
    # library picks for a lone instance (the cluster path, several steps per launch)
    for name, path in (("alone_generic", sgep.SGEP_PATH_GENERIC), ("alone_auto", sgep.SGEP_PATH_AUTO)):
        total_ms, steps, paths = 0.0, [], set()
        for i in range(n):
            s_ = mk(i, path)
            paths.add(s_.path)
            X, Y = pools[i]
            tt, ms_i, hit = 0, 0.0, None
            while tt < max_steps:
                e0.record()
                u = tt
                while u < tt + every:  # runs of consecutive minibatches within an epoch
                    m = min(tt + every - u, nmb - u % nmb)
                    o = offset(u)
                    s_.step_many(X[o:o + m * b], Y[o:o + m * b], b, m)
                    u += m
                e1.record()
                torch.cuda.synchronize()
                ms_i += e0.elapsed_time(e1)
                tt += every
                if err(i, s_) <= target:
                    hit = tt
                    break
            s_.close()
            steps.append(hit)
            total_ms += ms_i
        out[name] = {"paths": sorted(paths), "reached": sum(h is not None for h in steps),
                     "device_seconds_all_instances": total_ms / 1e3, "steps_per_instance": steps}
    bs = out["batched"]["device_seconds_to_all"]
    out["time_to_target_ratio"] = {k_: out[k_]["device_seconds_all_instances"] / bs for k_ in
                                   ("alone_generic", "alone_auto")}
    torch.cuda.empty_cache()
    return out


def planted_cca_truth(model, k):
    """Population top-k solution of the planted CCA model with orthonormal mixing columns
    (Qx, Qy), latent scales s and isotropic noise sigma: Cxx = Qx S^2 Qx^T + sigma^2 I,
    Cxy = Qx S^2 Qy^T. In the bases Qx, Qy every block is diagonal, so the pencil's top
    vectors are v_i = [Qx e_i; Qy e_i] / sqrt(2) with lambda_i = s_i^2 / (s_i^2 + sigma^2).
    Returns (V*, lambda, B-apply)."""
    s2, n2 = model.s ** 2, model.sigma ** 2
    Vt = np.concatenate([model.Qx[:, :k], model.Qy[:, :k]]) / np.sqrt(2.0)
    dx = model.d_x

    def Bmv(U):
        ux, uy = U[:dx], U[dx:]
        return np.concatenate([model.Qx @ (s2[:, None] * (model.Qx.T @ ux)) + n2 * ux,
                               model.Qy @ (s2[:, None] * (model.Qy.T @ uy)) + n2 * uy])
    return Vt, s2[:k] / (s2[:k] + n2), Bmv


def measure_warm_c5(dev, seed=0, n_train=3000, n_heldout=1096, n_tte=16, train_iters=300, slice_=250,
                    max_steps=40_000, check_every=512, per=128, target=1e-3):
    """Learned warm start at full size: 4096 CCA instances with d_x = d_y = 1024, k = 16 (mixing
    a smooth function of theta in [-1, 1]^8, 16 latent directions, correlations 0.9..0.3), the
    sketch of a 2048-row first minibatch, the per-row MLP trained on n_train instances, evaluated
    on n_heldout. Targets are the plain solver's fixed point, the population solution (closed
    form); the cold runs below reach it to 1e-3. Time to 1e-3 runs on the first n_tte held-out
    instances, warm and cold from the same fresh samples (b = 2048 per step, generated outside the
    timed region) with the same schedule and the same step cap."""
    import torch
    from paper_2206_04993_gb300 import Solver, WarmStart, sgep
    fam = synth.config_c5(seed=seed + 1)
    dx, k, b = fam["d_x"], fam["k"], 2048
    d = 2 * dx
    om = torch.tensor(fam["omega"], dtype=torch.float32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def sketch_of(model, rseed):
        X, Y = make_pool({"model": model}, b, "f32", dev, seed=rseed)
        return WarmStart.sketch(X, Y, om)

    t_data = time.time()
    sk, tg = [], []
    for i, th in enumerate(fam["thetas"](n_train, 0)):
        m = fam["model"](th)
        sk.append(sketch_of(m, 200_000 + i))
        tg.append(torch.tensor(planted_cca_truth(m, k)[0], dtype=torch.float32, device=dev))
    S, V = torch.cat(sk), torch.cat(tg)
    del sk, tg
    torch.cuda.synchronize()
    t_data = time.time() - t_data
    ws = WarmStart(m=16, k=k, seed=seed + 3)
    seg_all = [j * d for j in range(n_train + 1)]
    first = ws.loss_grad(S, V, seg_all)
    e0.record()
    for it in range(train_iters):
        i0 = (it * slice_) % n_train
        i1 = min(n_train, i0 + slice_)
        ws.loss_grad(S[i0 * d:i1 * d], V[i0 * d:i1 * d], [j * d for j in range(i1 - i0 + 1)])
        ws.adam_step(3e-3)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    last = ws.loss_grad(S, V, seg_all)
    del S, V
    # held-out: V0 from the network, and the sketch itself as a 16-column V (its information limit)
    held = [fam["model"](th) for th in fam["thetas"](n_heldout, 1)]
    err_net, err_sketch, V0s, inf_ms = [], [], [], 0.0
    for i, m in enumerate(held):
        X, Y = make_pool({"model": m}, b, "f32", dev, seed=400_000 + i)
        torch.cuda.synchronize()
        e0.record()
        Sk = WarmStart.sketch(X, Y, om)
        O = ws.forward(Sk)
        e1.record()
        torch.cuda.synchronize()
        if i > 0:
            inf_ms += e0.elapsed_time(e1)
        Vt, _, Bmv = planted_cca_truth(m, k)
        o = O.double().cpu().numpy()
        o /= np.linalg.norm(o, axis=0, keepdims=True)
        err_net.append(gen_subspace_error_op(Vt, o, Bmv))
        err_sketch.append(gen_subspace_error_op(Vt, Sk.double().cpu().numpy(), Bmv))
        if i < n_tte:
            V0s.append(o.astype(np.float32))
    ws.close()
    rng_cold = [synth.random_unit_columns(d, k, seed=700 + i).astype(np.float32) for i in range(n_tte)]
    # hold 0.3 for 200 steps, then eta_t = 40 / (t + Delta): the best of eta t -> 20, 40, 80, 160
    eta0, t_c, c = 0.3, 200, 40.0
    delta = c / eta0 - t_c
    eta_T = eta0 * (t_c + delta) / (max_steps + delta)
    out = {"scale": f"full: d_x = d_y = {dx}, k = {k}, latent 16, sketch of {b} rows; {n_train} training "
                    f"instances, {n_heldout} held-out (initial error), first {n_tte} held-out run to {target}",
           "targets": "population solution of each instance (closed form), the plain solver's fixed point",
           "train": {"iters": train_iters, "instances_per_iter": slice_, "loss_first_last": [first, last],
                     "device_ms": train_ms, "data_seconds_host": t_data},
           "inference_device_ms_per_instance": inf_ms / max(1, n_heldout - 1),
           "initial_error_median": {"warm": float(np.median(err_net)), "sketch_itself": float(np.median(err_sketch))},
           "schedule": {"eta0": eta0, "t_c": t_c, "eta_t_late": f"{c} / (t + {delta:.1f})"},
           "target": target, "max_steps": max_steps}
    for name, starts in (("cold", rng_cold), ("warm", V0s)):
        runs = []
        for i in range(n_tte):
            m = held[i]
            Vt, _, Bmv = planted_cca_truth(m, k)
            s = Solver(kind=sgep.SGEP_CCA, d_x=dx, d_y=dx, k=k, eta0=eta0, gamma0=0.3, rho=1e-6, schedule=1,
                       t_c=t_c, T=max_steps, eta_T=eta_T, max_b=b, seed=seed)
            s.set_V(starts[i])
            err0 = gen_subspace_error_op(Vt, starts[i].astype(np.float64), Bmv)
            t, ms, hit = 0, 0.0, None
            while t < max_steps:
                X, Y = make_pool({"model": m}, b * per, "f32", dev, seed=500_000 + 1000 * i + t // per)
                torch.cuda.synchronize()
                e0.record()
                s.step_many(X, Y, b, per)
                e1.record()
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                t += per
                del X, Y
                if t % check_every == 0 and gen_subspace_error_op(Vt, s.V().astype(np.float64), Bmv) <= target:
                    hit = t
                    break
            runs.append({"initial_error": round(err0, 4), "steps": hit, "device_seconds": ms / 1e3 if hit else None,
                         "path": s.path})
            s.close()
        steps = sorted(r["steps"] if r["steps"] else np.inf for r in runs)
        secs = sorted(r["device_seconds"] if r["device_seconds"] else np.inf for r in runs)
        med = lambda v: float(np.median(v)) if np.isfinite(np.median(v)) else None
        out[name] = {"reached": sum(r["steps"] is not None for r in runs), "of": n_tte,
                     "median_steps_to_target": med(steps), "median_device_seconds_to_target": med(secs),
                     "runs": runs}
    torch.cuda.empty_cache()
    return out


def measure_c3_error(dev, rank, steps=512, eta=1e3, per=16, every=64, rr_every=128, eval_rows=8192):
    """Error against device time on the activation-like workload (d = 32768, k = 32, b = 4096):
    plain FP32 rows (tensor-core path, rows split into BF16 pairs), BF16 rows (streamed
    tensor-core steps) and BF16 rows with a
    Rayleigh-Ritz correction every rr_every steps, from the same random V on the same fresh
    samples (per minibatches drawn at a time, BF16 forms reading the rounded values), the same
    constant step size. Errors: generalized subspace error against the population solution
    (closed form) and the largest |Rayleigh quotient - canonical correlation| on an evaluation
    batch. 1e-3 is out of reach at this size within the configured 10M samples (top-32 gap about
    0.01); the curves show that the forms make the same progress per step."""
    import torch
    from paper_2206_04993_gb300 import Solver, sgep
    cfg = synth.config_c3(seed=rank)
    model = cfg["model"]
    b, k = cfg["b"], cfg["k"]
    Vt, lam, Bmv = lowrank_cca_truth(model, k)
    V0 = synth.random_unit_columns(model.d_x + model.d_y, k, seed=rank + 1).astype(np.float32)
    Xe, Ye = make_pool(cfg, eval_rows, "bf16", dev, seed=rank + 9999)
    out = {"steps": steps, "eta": eta, "samples_per_step": b, "truth": "population closed form (Woodbury)",
           "canonical_correlations": [round(float(lam[0]), 4), round(float(lam[-1]), 4)]}
    forms = (("f32", "f32", 0), ("bf16", "bf16", 0), ("bf16_rr", "bf16", rr_every))
    for name, dt, rr in forms:
        s = Solver(kind=sgep.SGEP_CCA, d_x=model.d_x, d_y=model.d_y, k=k,
                   dtype=sgep.SGEP_BF16 if dt == "bf16" else sgep.SGEP_F32, eta0=eta, gamma0=0.3,
                   rho=cfg["rho"], max_b=max(b, eval_rows), seed=rank)
        s.set_V(V0)
        if rr:
            s.set_rr_every(rr, Xe, Ye)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        curve, ms, t = [(0, 0.0, round(gen_subspace_error_op(Vt, V0.astype(np.float64), Bmv), 6))], 0.0, 0
        while t < steps:
            X, Y = make_pool(cfg, b * per, dt, dev, seed=rank + 10 + t // per)
            torch.cuda.synchronize()
            e0.record()
            s.step_many(X, Y, b, per)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            t += per
            del X, Y
            if t % every == 0:
                curve.append((t, round(ms / 1e3, 5), round(gen_subspace_error_op(Vt, s.V().astype(np.float64), Bmv), 6)))
        lam_hat = s.eigenvalues(Xe if dt == "bf16" else Xe.float(), Ye if dt == "bf16" else Ye.float())
        out[name] = {"path": s.path, "device_seconds": ms / 1e3, "ms_per_step": ms / steps,
                     "curve_steps_seconds_error": curve, "final_error": curve[-1][2],
                     "max_eigenvalue_error": float(np.max(np.abs(np.sort(lam_hat)[::-1] - lam)))}
        s.close()
        torch.cuda.empty_cache()
    # device time of each form to the error level the plain FP32 form reaches at the end
    target = out["f32"]["final_error"]
    for name in ("f32", "bf16", "bf16_rr"):
        hit = [c for c in out[name]["curve_steps_seconds_error"][1:] if c[2] <= target]
        out[name]["seconds_to_f32_final_error"] = hit[0][1] if hit else None
    return out


def measure_tte(dev, rank, args):
    """Time to 1e-3 generalized subspace error on the 1024-dim FP32 workload (1,000,000-row
    resident pool), plain FP32 rows against the same rows in BF16, three initial V each."""
    import torch
    from paper_2206_04993_gb300 import Solver, sgep
    name, _, pool_rows = WORKLOADS[TTE_WORKLOAD]
    cfg = getattr(synth, name)(seed=rank)
    model = cfg["model"]
    b, k = cfg["b"], cfg["k"]
    dx, dy = model.d_x, model.d_y
    X, Y = make_pool(cfg, pool_rows, "f32", dev, seed=rank)
    truth = pool_truth(X, Y, k)

    def mk(dt):
        return lambda: Solver(kind=sgep.SGEP_CCA, d_x=dx, d_y=dy, k=k,
                              dtype=sgep.SGEP_BF16 if dt == "bf16" else sgep.SGEP_F32,
                              eta0=cfg["eta0"], gamma0=cfg["gamma0"], rho=cfg["rho"],
                              schedule=cfg["schedule"], t_c=cfg["t_c"], T=cfg["T"],
                              eta_T=cfg["eta_T"], max_b=b, path=args.path, seed=rank)

    def median_runs(fn):
        runs = [fn(seed) for seed in (1, 2, 3)]
        secs = sorted(r["seconds"] if r["reached"] else float("inf") for r in runs)
        steps = sorted(r["steps"] if r["reached"] else 10 ** 12 for r in runs)
        return {"median_seconds": secs[1], "median_steps": steps[1] if steps[1] < 10 ** 12 else None,
                "reached": sum(r["reached"] for r in runs), "runs": [
                    {kk: r[kk] for kk in ("reached", "steps", "seconds", "final_error")} for r in runs],
                "curve_seed1": runs[0]["curve"]}
    tte = {"workload": TTE_WORKLOAD,
           "truth": "scipy eigh of the pool's FP64 covariances (the paper's ground truth, Sec. 5)",
           "seeds": "initial V from seeds 1, 2, 3; median reported; device time of the steps only",
           "plain_f32": median_runs(lambda sd: time_to_error(mk("f32"), X, Y, b, truth, every=1000,
                                                             max_steps=args.tte_max_steps, seed=sd))}
    Xb, Yb = X.to(torch.bfloat16), Y.to(torch.bfloat16)
    tte["bf16"] = median_runs(lambda sd: time_to_error(mk("bf16"), Xb, Yb, b, truth, every=1000,
                                                       max_steps=args.tte_max_steps, seed=sd))
    del X, Y, Xb, Yb
    torch.cuda.empty_cache()
    return tte


def cpu_cores():
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    name, _, pool_rows = WORKLOADS[args.workload]
    if args.pool_rows:
        pool_rows = args.pool_rows
    cfg = getattr(synth, name)()
    # a bounded sample: about 0.5 s of oracle work per requested step, 5 s to 60 s in total
    rate, steps, el = oracle_rate(cfg, min(60.0, max(5.0, 0.5 * args.steps)))
    sample = f"{steps} oracle steps of b={cfg['b']} rows ({el:.1f} s), FP64 numpy, streamed operators"
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic planted CCA",
        "config": line_config(args.workload, pool_rows, world),
        "cpu_baseline": {"value": rate, "unit": "samples/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------

def run_native(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2206_04993_gb300 import Solver, sgep

    name, dtype, pool_rows = WORKLOADS[args.workload]
    if args.pool_rows:
        pool_rows = args.pool_rows
    cfg = getattr(synth, name)(seed=rank)
    model = cfg["model"]
    b, k = cfg["b"], cfg["k"]
    dx, dy = model.d_x, model.d_y
    d = dx + dy
    esz = 2 if dtype == "bf16" else 4
    X, Y = make_pool(cfg, pool_rows, dtype, dev, seed=rank)
    nb = pool_rows // b
    solver = Solver(kind=sgep.SGEP_CCA, d_x=dx, d_y=dy, k=k,
                    dtype=sgep.SGEP_BF16 if dtype == "bf16" else sgep.SGEP_F32,
                    eta0=cfg["eta0"], gamma0=cfg["gamma0"], rho=cfg["rho"],
                    schedule=cfg["schedule"], t_c=cfg["t_c"], T=cfg["T"], eta_T=cfg["eta_T"],
                    max_b=b, path=args.path, seed=rank)
    stream = torch.cuda.current_stream()

    def run_steps(start, count):
        s = start
        left = count
        while left > 0:
            j = s % nb
            n = min(left, nb - j)
            solver.step_many(X[j * b:(j + n) * b], Y[j * b:(j + n) * b], b, n)
            s += n
            left -= n
        return s

    pos = run_steps(0, args.warmup)
    solver.sync()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = solver.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        pos = run_steps(pos, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = solver.launches - launches0
    ms = world_max(ev0.elapsed_time(ev1), world, dev)
    solver.sync()
    ms_step = ms / args.steps
    value = world * b * args.steps / (ms / 1e3)

    # roofline of the step (the minibatch is read once; V and [Bv] are read and written once).
    # On the streamed tensor-core path and the cluster path the timed steps are exactly the
    # launches of one kernel (the streamed kernel runs every step of a step_many call, the
    # cluster kernel one step per launch), so the step time is that kernel's time per step.
    peak, peak_kind = measured_peaks()
    alg_bytes = b * d * esz + 16 * d * k
    achieved = alg_bytes / (ms_step / 1e3) / 1e9
    kernels = {sgep.SGEP_PATH_CLUSTER: "k_cluster_step (one step per launch)",
               sgep.SGEP_PATH_TC: "k_tc_stream (products, row-side terms and update of every step of a "
                                  "step_many call in one launch)"}
    one_kernel = solver.path in kernels and launches <= -(-args.steps // max(1, min(nb, 64)))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": TRAFFIC_BYTES.get(args.workload) if one_kernel else None,
                "traffic_unit": "DRAM bytes read + written per step (one ncu capture)",
                "kernel": kernels[solver.path] if one_kernel else f"whole step, path {solver.path}",
                "peak_source": peak_kind, "alg_bytes_per_step": alg_bytes,
                "alg_bytes_formula": "b d (element bytes) + 16 d k",
                "timing": "CUDA events over the timed launches on their stream (the step's only kernel)"
                if one_kernel else "CUDA events over the timed launches on their stream"}

    # e2e: through the C ABI with host buffers every step
    e2e = None
    if not args.no_e2e:
        ne = min(args.steps, 200)
        Xh = torch.empty((4, b, dx), dtype=X.dtype, pin_memory=True)
        Yh = torch.empty((4, b, dy), dtype=Y.dtype, pin_memory=True)
        for i in range(4):
            Xh[i].copy_(X[i * b:(i + 1) * b])
            Yh[i].copy_(Y[i * b:(i + 1) * b])
        # two device buffers: the copies of step i + 1 (X and Y on their own copy streams) run
        # while step i computes; every step's V is read back to the host before the next step
        Xd = [torch.empty((b, dx), dtype=X.dtype, device=dev) for _ in range(2)]
        Yd = [torch.empty((b, dy), dtype=Y.dtype, device=dev) for _ in range(2)]
        cs = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]
        ready = [[torch.cuda.Event(), torch.cuda.Event()] for _ in range(2)]
        freed = [torch.cuda.Event(), torch.cuda.Event()]
        Vh = np.empty((d, k), dtype=np.float32)

        def issue_copy(i):
            u = i % 2
            for which, (dst, src) in enumerate(((Xd[u], Xh[i % 4]), (Yd[u], Yh[i % 4]))):
                with torch.cuda.stream(cs[which]):
                    if i >= 2:
                        cs[which].wait_event(freed[u])  # the step that read this buffer is done
                    dst.copy_(src, non_blocking=True)
                    ready[u][which].record(cs[which])

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        issue_copy(0)
        for i in range(ne):
            u = i % 2
            stream.wait_event(ready[u][0])
            stream.wait_event(ready[u][1])
            solver.step(Xd[u], Yd[u])
            freed[u].record(stream)
            if i + 1 < ne:
                issue_copy(i + 1)
            sgep.sgep_get_V(solver.h, Vh, False, stream.cuda_stream)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e = {"value": world * b * ne / el, "unit": "samples/s",
               "h2d_bytes_per_step": b * d * esz, "d2h_bytes_per_step": d * k * 4,
               "steps": ne}

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, steps, el = oracle_rate(cfg, args.cpu_seconds)
        cpu = {"value": rate, "unit": "samples/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{steps} FP64 oracle steps of b={b} ({el:.1f} s) on this workload"}

    forms = None
    if rank == 0 and not args.no_forms:
        del X, Y
        torch.cuda.empty_cache()
        forms = {}
        if args.workload != TTE_WORKLOAD:
            forms[TTE_WORKLOAD] = measure_throughput(TTE_WORKLOAD, 2000, 20, dev, rank)
        if not args.no_tte:
            forms[TTE_WORKLOAD + "_time_to_1e-3"] = measure_tte(dev, rank, args)
            forms["cca_d32768_k32_b4096_error_vs_time"] = measure_c3_error(dev, rank)
        if args.workload != "cca_d32768_k32_b4096_f32":
            # the plain FP32 form of the same problem
            forms["cca_d32768_k32_b4096_f32"] = measure_throughput("cca_d32768_k32_b4096_f32", 8, 3, dev, rank)
            # the same FP32 rows on the generic SIMT path (register-tiled FMA contractions)
            forms["cca_d32768_k32_b4096_f32_simt"] = measure_throughput("cca_d32768_k32_b4096_f32", 8, 3, dev, rank,
                                                                        path=1)
        if args.workload == "cca_d32768_k32_b4096_bf16":
            forms["bf16_vs_f32_step_speedup_d32768"] = forms["cca_d32768_k32_b4096_f32"]["ms_per_step"] / ms_step
        forms["batch64_cca_lda_b512_f32"] = measure_batch("f32", 40, 3, dev, seed=rank)
        forms["batch64_cca_lda_b512_bf16"] = measure_batch("bf16", 40, 3, dev, seed=rank)
        forms["warm_start_cca_family"] = measure_warm(dev, seed=rank)
        if not args.no_tte:
            forms["batch16_cca_time_to_1e-3"] = measure_batch_tte(dev, seed=rank)
        if not args.no_tte:
            forms["warm_start_c5"] = measure_warm_c5(dev, seed=rank)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic planted CCA generated on device",
            "config": line_config(args.workload, pool_rows, world), "path": solver.path,
            "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk.summary(), "forms": forms,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
