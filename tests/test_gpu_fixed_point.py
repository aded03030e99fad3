"""GPU dust-temperature fixed point against the oracle's (marked gpu)."""
import numpy as np
import pytest

import synth
from gpu_util import build_ctx

pytestmark = pytest.mark.gpu


def _gpu_fp(w, unroll, tol=1e-4):
    import torch
    ctx, _ = build_ctx(w)
    td = torch.as_tensor(w.td, device="cuda:0").clone()
    tg = torch.as_tensor(w.tgas, device="cuda:0")
    it = ctx.fixed_point(tg, td, max_iter=60, tol=tol, unroll=unroll)
    ctx.check()
    return td.cpu().numpy(), it


@pytest.mark.parametrize("unroll", [0, 4])
def test_fixed_point_matches_oracle(orc, unroll):
    w = synth.with_gas(synth.turbulent_cloud(32), seed=7)
    ref, it_ref, _ = orc.fixed_point(w, w.tgas, w.td, max_iter=60, tol=1e-4)
    td, it = _gpu_fp(w, unroll)
    assert it_ref > 0 and abs(it - it_ref) <= 1, (it, it_ref)
    assert np.abs(td / ref - 1).max() < 1e-4


def test_graph_equals_plain_loop():
    w = synth.with_gas(synth.turbulent_cloud(32), seed=7)
    a, ia = _gpu_fp(w, 0)
    b, ib = _gpu_fp(w, 3)
    assert ia == ib
    assert np.abs(a / b - 1).max() < 1e-5


def test_refresh_equals_rebuild():
    """treeray_refresh with new T_d gives the same moments as a full rebuild."""
    import torch
    w = synth.turbulent_cloud(16)
    ctx, t = build_ctx(w)
    td2 = (t["td"] * 1.3 + 2.0).contiguous()
    ctx.refresh(td2)
    ctx.check()
    a = ctx.tree_export()
    w2 = synth.turbulent_cloud(16)
    w2.td = td2.cpu().numpy()
    ctx2, _ = build_ctx(w2)
    b = ctx2.tree_export()
    assert np.array_equal(a["vals"], b["vals"])
