"""Dust temperature (Sec. 4.6, App. D) on many cells spanning wide ranges of density, gas
temperature, radiation field and extra heating, against the oracle's bisection.

The GPU locates the root in FP32 and decides the FP32 result in FP64; the oracle bisects
in FP64. Both round the same root, so they agree except where the root lies within an
FP64 rounding of the midpoint between two floats (one unit in the last place)."""
import numpy as np
import pytest

import synth
from gpu_util import build_ctx

pytestmark = pytest.mark.gpu


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    rho = (10.0 ** rng.uniform(-26, -14, n)).astype(np.float32)
    tgas = (10.0 ** rng.uniform(np.log10(2.0), np.log10(3000.0), n)).astype(np.float32)
    J = (10.0 ** rng.uniform(-12, 6, n)).astype(np.float32)
    J[rng.random(n) < 0.02] = 0.0
    heat = np.where(rng.random(n) < 0.3, 10.0 ** rng.uniform(-30, -18, n), 0.0).astype(np.float32)
    kap = (10.0 ** rng.uniform(-2, 1.5, n)).astype(np.float32)
    return rho, tgas, J, heat, kap


@pytest.mark.parametrize("mode", ["grey", "planck", "given"])
def test_dust_temperature_wide_ranges(orc, mode):
    import torch
    n = 32
    w = synth.homogeneous(n, 1.0, 1e-20, td=20.0, kappa0=5.0)
    rho, tgas, J, heat, kap = _inputs(w.n_leaves, {"grey": 1, "planck": 2, "given": 3}[mode])
    w.rho = rho
    w.params = dict(w.params, kappa_model=1 if mode == "planck" else 0)
    w.kappa = kap if mode == "given" else None
    ctx, _ = build_ctx(w)
    dev = "cuda:0"
    Td = torch.empty(w.n_leaves, dtype=torch.float32, device=dev)
    ctx.dust_temperature(torch.as_tensor(tgas, device=dev), torch.as_tensor(J, device=dev), Td,
                         heat_extra=torch.as_tensor(heat, device=dev))
    ctx.check()
    Tg = Td.cpu().numpy()
    Tr = orc.dust_temperature(w.params, rho, tgas, J.astype(np.float64), heat,
                              kappa=kap if mode == "given" else None).astype(np.float32)
    rel = np.abs(Tg.astype(np.float64) / Tr - 1.0)
    assert rel.max() <= 2e-7, (rel.max(), np.argmax(rel))
    assert np.mean(Tg == Tr) >= 0.999
