"""Helpers for the GPU tests: build a library context from a synthetic workload."""
import numpy as np


def build_ctx(w, params=None, stream=None):
    import torch

    import paper_2204_09072_gb300 as tr
    p = dict(w.params if params is None else params)
    ctx = tr.Context(p)
    dev = torch.device("cuda:0")
    rho = torch.from_numpy(np.ascontiguousarray(w.rho, np.float32)).to(dev)
    td = torch.from_numpy(np.ascontiguousarray(w.td, np.float32)).to(dev)
    kap = None if w.kappa is None else torch.from_numpy(np.ascontiguousarray(w.kappa, np.float32)).to(dev)
    ctx.build(w.box_cm, rho, td, n=w.uniform_n, blocks=w.blocks, kappa=kap,
              star_pos=w.star_pos if len(w.star_lum) else None,
              star_lum=w.star_lum if len(w.star_lum) else None, stream=stream)
    ctx.check(stream)
    return ctx, dict(rho=rho, td=td, kappa=kap)


def evaluate(ctx, targets=None, stream=None):
    import torch
    dev = torch.device("cuda:0")
    n = ctx.leaf_count if targets is None else len(targets)
    J = torch.empty(n, dtype=torch.float32, device=dev)
    F = torch.empty(n * 3, dtype=torch.float64, device=dev)
    t = None if targets is None else torch.as_tensor(np.asarray(targets), dtype=torch.int32, device=dev)
    ctx.evaluate(J, F, targets=t, stream=stream)
    ctx.check(stream)
    return J.cpu().numpy().astype(np.float64), F.cpu().numpy().reshape(n, 3)


def flux_err(F, Fr, J):
    """|dF| / max(|F_ref|, 1e-2 x 4 pi J): the 48-ray sum cancels, so |F| can be tiny."""
    den = np.maximum(np.linalg.norm(Fr, axis=1), 1e-2 * 4 * np.pi * J)
    return np.linalg.norm(F - Fr, axis=1) / den
