"""Learned warm start on the GPU: the sketch, the network's forward pass, loss and
gradients against the oracle (oracle/warm.py), and what a trained network gains over
the plain cold-started iteration on held-out instances of a planted family."""
import numpy as np
import pytest

import synth
from gpu_util import bf16_round, rel, to_device
from oracle import gep, warm
from paper_2206_04993_gb300 import sgep as S

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("dx,dy,n,dtype", [(40, 24, 300, "f32"), (128, 0, 500, "f32"), (96, 96, 700, "bf16")],
                         ids=["two_view", "one_view", "bf16"])
def test_sketch_matches_oracle(dx, dy, n, dtype):
    from paper_2206_04993_gb300 import WarmStart
    rng = np.random.default_rng(0)
    X = rng.standard_normal((n, dx)) * np.linspace(2.0, 0.5, dx)
    Y = None if dy == 0 else 0.5 * X[:, :dy] + rng.standard_normal((n, dy))
    if dtype == "bf16":
        X = bf16_round(X)
        Y = None if Y is None else bf16_round(Y)
    om = rng.standard_normal((dx + dy, 16)).astype(np.float32)
    Sg = WarmStart.sketch(to_device(X, dtype), None if Y is None else to_device(Y, dtype), _dev(om),
                          dtype=S.SGEP_BF16 if dtype == "bf16" else S.SGEP_F32).cpu().numpy()
    Sr = warm.sketch(np.asarray(X, np.float32), None if Y is None else np.asarray(Y, np.float32), om)
    assert rel(Sg, Sr) < 1e-5


def _random_params(ws, rng):
    p = rng.standard_normal(ws.P).astype(np.float32) * 0.2
    ws.set_params(p)
    return ws.params()


def _split(p, m, k):
    H = 64
    o = np.cumsum([0, H * m, H, H * H, H, k * H, k])
    return [p[o[0]:o[1]].reshape(H, m), p[o[1]:o[2]], p[o[2]:o[3]].reshape(H, H), p[o[3]:o[4]],
            p[o[4]:o[5]].reshape(k, H), p[o[5]:o[6]]]


def test_forward_matches_oracle():
    from paper_2206_04993_gb300 import WarmStart
    rng = np.random.default_rng(1)
    ws = WarmStart(m=16, k=7, seed=3)
    p = _random_params(ws, rng)
    Sx = rng.standard_normal((1000, 16)).astype(np.float32)
    out = ws.forward(_dev(Sx)).cpu().numpy()
    ref, _ = warm.forward(_split(p, 16, 7), Sx)
    assert rel(out, ref) < 1e-5
    # the weights in use are BF16 values, the biases FP32
    H = 64
    assert np.all(_split(p, 16, 7)[0] == bf16_round(_split(p, 16, 7)[0]))
    ws.close()


def test_loss_and_gradients_match_oracle():
    from paper_2206_04993_gb300 import WarmStart
    rng = np.random.default_rng(2)
    m, k = 12, 5
    ws = WarmStart(m=m, k=k, seed=4)
    p = _random_params(ws, rng)
    seg = [0, 300, 420, 1000]
    Sx = rng.standard_normal((1000, m)).astype(np.float32)
    V = rng.standard_normal((1000, k)).astype(np.float32)
    loss, g = ws.loss_grad(_dev(Sx), _dev(V), seg, grads=True)
    params = _split(p, m, k)
    Sl = [Sx[seg[i]:seg[i + 1]] for i in range(3)]
    Vl = [V[seg[i]:seg[i + 1]] for i in range(3)]
    loss_r, grads_r = warm.loss_and_grads(params, Sl, Vl)
    assert abs(loss - loss_r) <= 1e-5 * abs(loss_r)
    for name, a, b in zip(["W1", "b1", "W2", "b2", "W3", "b3"], _split(g, m, k), grads_r):
        assert rel(a, b) < 1e-4, (name, rel(a, b))
    ws.close()


def test_trained_network_beats_cold_start():
    """Train on the plain solver's solutions of 192 planted instances, then start 16 held-out
    instances from the network's V0: lower error at the start and after 100 steps."""
    import torch
    from paper_2206_04993_gb300 import Batch, Solver, WarmStart
    fam = synth.config_c5(seed=1, d_x=64, k=4, latent=8, spread=0.3)
    k, d_x = 4, 64
    d = 2 * d_x
    om = _dev(fam["omega"])
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(5)

    def rows(model, n):
        Wx = torch.tensor(model.Qx * model.s, dtype=torch.float32, device=dev)
        Wy = torch.tensor(model.Qy * model.s, dtype=torch.float32, device=dev)
        z = torch.randn(n, model.s.size, device=dev, generator=g)
        return (z @ Wx.T + 0.5 * torch.randn(n, d_x, device=dev, generator=g),
                z @ Wy.T + 0.5 * torch.randn(n, d_x, device=dev, generator=g))

    def sketches(models):
        out = []
        for mdl in models:
            X, Y = rows(mdl, 2048)
            out.append(WarmStart.sketch(X, Y, om))
        return out

    def solve(models, steps, V0=None, b=512):
        ss = [Solver(kind=S.SGEP_CCA, d_x=d_x, d_y=d_x, k=k, max_b=b, path=S.SGEP_PATH_GENERIC, eta0=0.1,
                     gamma0=0.3, seed=100 + i) for i in range(len(models))]
        if V0 is not None:
            for s, v in zip(ss, V0):
                s.set_V(v)
        with Batch(ss) as bt:
            for t in range(steps):
                data = [rows(mdl, b) for mdl in models]
                bt.step([x for x, _ in data], [y for _, y in data], [b] * len(models))
            bt.sync()
        Vs = [s.V().astype(np.float64) for s in ss]
        for s in ss:
            s.close()
        return Vs

    def errors(models, Vs):
        out = []
        for mdl, V in zip(models, Vs):
            _, Vt = gep.cca_truth_planted(mdl, k)
            out.append(gep.subspace_error(Vt, V, lambda U, mdl=mdl: gep.cca_B_apply(mdl, U)))
        return np.array(out)

    train = [fam["model"](t) for t in fam["thetas"](192, 0)]
    held = [fam["model"](t) for t in fam["thetas"](16, 1)]
    V_train = solve(train, 1500)
    assert np.median(errors(train, V_train)) < 0.05  # the targets are converged solutions
    S_train = torch.cat(sketches(train))
    T_train = _dev(np.concatenate(V_train))
    seg = [i * d for i in range(len(train) + 1)]
    ws = WarmStart(m=16, k=k, seed=7)
    first = ws.loss_grad(S_train, T_train, seg)
    for it in range(400):
        loss = ws.loss_grad(S_train, T_train, seg)
        ws.adam_step(3e-3)
    assert loss < 0.5 * first, (first, loss)
    V0 = []
    for Sk in sketches(held):
        v = ws.forward(Sk).cpu().numpy().astype(np.float64)
        V0.append((v / np.linalg.norm(v, axis=0)).astype(np.float32))
    cold0 = errors(held, [synth.random_unit_columns(d, k, seed=100 + i) for i in range(len(held))])
    warm0 = errors(held, V0)
    warm100 = errors(held, solve(held, 100, V0=V0))
    cold100 = errors(held, solve(held, 100))
    print("start", cold0.mean(), warm0.mean(), "after 100", cold100.mean(), warm100.mean(), "loss", first, loss)
    assert warm0.mean() < 0.5 * cold0.mean()
    assert warm100.mean() < cold100.mean()
    ws.close()


def test_full_size_family_trained_network_reaches_the_sketch_limit():
    """The full-size family (d_x = d_y = 1024, k = 16, 2048-row sketch), trained on 3000
    instances with the population solutions as targets: on 16 held-out instances the network's
    V0 has a lower generalized subspace error than a random start and is within 0.03 of the
    error of the sketch's own 16 columns (the information the network's input carries)."""
    import torch
    from paper_2206_04993_gb300 import WarmStart
    fam = synth.config_c5(seed=1)
    d_x, k = fam["d_x"], fam["k"]
    d = 2 * d_x
    om = _dev(fam["omega"])
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(11)

    def sketch(model):
        Wx = torch.tensor(model.Qx * model.s, dtype=torch.float32, device=dev)
        Wy = torch.tensor(model.Qy * model.s, dtype=torch.float32, device=dev)
        z = torch.randn(2048, model.s.size, device=dev, generator=g)
        X = z @ Wx.T + model.sigma * torch.randn(2048, d_x, device=dev, generator=g)
        Y = z @ Wy.T + model.sigma * torch.randn(2048, d_x, device=dev, generator=g)
        return WarmStart.sketch(X, Y, om)

    def error(model, V):
        _, Vt = gep.cca_truth_planted(model, k)
        return gep.subspace_error(Vt, V, lambda U: gep.cca_B_apply(model, U))

    sk, tg = [], []
    for th in fam["thetas"](3000, 0):
        mdl = fam["model"](th)
        sk.append(sketch(mdl))
        tg.append(_dev(gep.cca_truth_planted(mdl, k)[1]))
    S_all, T_all = torch.cat(sk), torch.cat(tg)
    del sk, tg
    ws = WarmStart(m=16, k=k, seed=3)
    seg = [i * d for i in range(3001)]
    first = ws.loss_grad(S_all, T_all, seg)
    for it in range(300):
        i0 = (it * 250) % 3000
        ws.loss_grad(S_all[i0 * d:(i0 + 250) * d], T_all[i0 * d:(i0 + 250) * d], [j * d for j in range(251)])
        ws.adam_step(3e-3)
    last = ws.loss_grad(S_all, T_all, seg)
    assert last < first, (first, last)
    held = [fam["model"](th) for th in fam["thetas"](16, 1)]
    warm, limit, cold = [], [], []
    for i, mdl in enumerate(held):
        Sk = sketch(mdl)
        warm.append(error(mdl, ws.forward(Sk).cpu().numpy().astype(np.float64)))
        limit.append(error(mdl, Sk.cpu().numpy().astype(np.float64)))
        cold.append(error(mdl, synth.random_unit_columns(d, k, seed=900 + i)))
    ws.close()
    print("loss", first, last, "median V0 error: warm", np.median(warm), "sketch", np.median(limit),
          "cold", np.median(cold))
    assert np.median(cold) > 0.95
    assert np.median(warm) < 0.85
    assert np.median(warm) < np.median(limit) + 0.03
