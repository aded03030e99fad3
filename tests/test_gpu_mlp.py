"""Warm-start network on the GPU against the FP64 reference (marked gpu)."""
import numpy as np
import pytest

import synth
from gpu_util import build_ctx
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _random_net(seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.25, omlp.N_PARAMS).astype(np.float32)
    norm = np.concatenate([rng.normal(0, 1, 6), rng.uniform(0.5, 2, 6), [1.2, 0.4]]).astype(np.float32)
    return p, norm


def _data(seed, n, norm):
    rng = np.random.default_rng(seed)
    X = (rng.normal(0, 1, (n, 6)) * norm[6:12] + norm[0:6]).astype(np.float32)
    y = rng.normal(1.2, 0.4, n).astype(np.float32)
    return X, y


def test_gradient_matches_reference():
    import torch

    import paper_2204_09072_gb300 as tr
    p, norm = _random_net(1)
    X, y = _data(2, 512, norm)
    net = tr.MLP(seed=5)
    net.set_params(p, norm)
    g, loss = net.grad(torch.as_tensor(X.reshape(-1), device="cuda:0"), torch.as_tensor(y, device="cuda:0"))
    lref, gref = omlp.loss_and_grad(p, norm, X, y, bf16=True)
    assert abs(loss - lref) <= 1e-4 * abs(lref)
    assert np.linalg.norm(g - gref) <= 2e-3 * np.linalg.norm(gref)
    for a, b in [(0, 384), (448, 4544), (4608, 4673)]:
        assert np.linalg.norm(g[a:b] - gref[a:b]) <= 5e-3 * np.linalg.norm(gref[a:b])


def test_tensor_core_inference_matches_reference():
    import torch

    import paper_2204_09072_gb300 as tr
    p, norm = _random_net(3)
    X, _ = _data(4, 1000, norm)  # not a multiple of the 16-row tile
    net = tr.MLP(seed=5)
    net.set_params(p, norm)
    yg = net.infer(torch.as_tensor(X.reshape(-1), device="cuda:0")).cpu().numpy()
    yr = omlp.predict_log10(p, norm, X, bf16=True)
    err = np.abs(yg - yr)
    assert err.max() <= 1e-2 * norm[13] and np.median(err) <= 1e-3 * norm[13]


def test_training_reduces_loss():
    import torch

    import paper_2204_09072_gb300 as tr
    rng = np.random.default_rng(7)
    X = rng.normal(0, 1, (16384, 6)).astype(np.float32)
    y = (1.3 + 0.3 * np.sin(X[:, 0]) + 0.2 * X[:, 1] * X[:, 2] / (1 + X[:, 3] ** 2)).astype(np.float32)
    Xt = torch.as_tensor(X.reshape(-1), device="cuda:0")
    yt = torch.as_tensor(y, device="cuda:0")
    net = tr.MLP(seed=9)
    net.fit_normalization(Xt, yt)
    hist = net.train(Xt, yt, steps=1500, batch=1024, lr=3e-3, seed=11)
    assert hist[-50:].mean() < 0.05 * hist[:10].mean()


def _solve(seed):
    import torch
    w = synth.with_gas(synth.turbulent_cloud(32, seed=seed), seed=seed + 1)
    ctx, t = build_ctx(w)
    tg = torch.as_tensor(w.tgas, device="cuda:0")
    X = ctx.features(tg)[0].clone()
    td = t["td"].clone()
    it = ctx.fixed_point(tg, td, tol=1e-4, max_iter=100)
    return ctx, tg, t["td"], X, td, it


def test_warm_start_cuts_iterations():
    import torch

    import paper_2204_09072_gb300 as tr
    Xs, ys = [], []
    for s in (21, 22, 23):
        _, _, _, X, td, _ = _solve(s)
        Xs.append(X)
        ys.append(torch.log10(td))
    X = torch.cat(Xs).reshape(-1).contiguous()
    y = torch.cat(ys).contiguous()
    net = tr.MLP(seed=4)
    net.fit_normalization(X, y)
    net.train(X, y, steps=2500, batch=2048, lr=2e-3, seed=3)
    ctx, tg, td0, Xn, td_plain, it_plain = _solve(31)
    td_warm = td0.clone()
    ctx.warm_start(net, Xn.reshape(-1).contiguous(), td_warm)
    guess = td_warm.clone()
    it_warm = ctx.fixed_point(tg, td_warm, tol=1e-4, max_iter=100)
    g_err = (guess / td_plain - 1).abs().max().item()
    d = (td_warm / td_plain - 1).abs().max().item()
    print(f"plain {it_plain} iterations, warm start {it_warm} (+1 feature pass); "
          f"guess max rel err {g_err:.2e}; converged max rel diff {d:.2e}")
    assert it_warm < it_plain
    assert d < 5e-4
