"""Batched evaluation, warps-per-target choices and the autotuner (marked gpu)."""
import numpy as np
import pytest

import synth
from gpu_util import build_ctx, evaluate, flux_err

pytestmark = pytest.mark.gpu


def _boxes():
    return [synth.gaussian_clump(16, nbins=16),
            synth.random_uniform(16, seed=21, thick_frac=0.1, nbins=16),
            synth.amr_core(n_base_blocks=2, max_level=1, target_leaves=12 * 512, n_stars=2, nbins=16),
            synth.turbulent_cloud(32, nbins=16),
            synth.point_source(8, kappa0=2.0, nbins=16)]


@pytest.mark.parametrize("use_graph,thin_wpt", [(False, 4), (True, 4), (True, 3), (True, 2), (False, 2)])
def test_batch_matches_single_and_oracle(orc, use_graph, thin_wpt):
    """Thin boxes run teams of the first thin box's size (2, 3 or 4 warps), thick boxes 4."""
    import torch

    import paper_2204_09072_gb300 as tr
    ws = _boxes()
    ctxs = [build_ctx(w)[0] for w in ws]
    for c in ctxs:
        c.set_warps_per_target(thin_wpt)
    singles = [evaluate(c) for c in ctxs]
    b = tr.Batch(ctxs)
    Js = [torch.empty(c.leaf_count, dtype=torch.float32, device="cuda:0") for c in ctxs]
    Fs = [torch.empty(3 * c.leaf_count, dtype=torch.float64, device="cuda:0") for c in ctxs]
    for _ in range(2):  # the second call replays the graph
        b.evaluate(Js, Fs, use_graph=use_graph)
    for c in ctxs:
        c.check()
    for w, c, (Js1, Fs1), J, F in zip(ws, ctxs, singles, Js, Fs):
        J = J.double().cpu().numpy()
        F = F.cpu().numpy().reshape(-1, 3)
        assert np.abs(J / Js1 - 1).max() < 1e-5
        assert flux_err(F, Fs1, Js1).max() < 1e-5
        tg = synth.sample_targets(w.n_leaves, 256, seed=2)
        Jr, Fr = orc.Tree(w).evaluate(tg)
        assert np.abs(J[tg] / Jr - 1).max() <= 1e-4
        assert flux_err(F[tg], Fr, Jr).max() <= 1e-4
    b.close()


@pytest.mark.parametrize("wpt,thick_frac", [(2, 0.1), (8, 0.1), (3, 0.0), (2, 0.0), (8, 0.0)])
def test_team_sizes_match_oracle(orc, wpt, thick_frac):
    w = synth.random_uniform(16, seed=13, thick_frac=thick_frac)
    ctx, _ = build_ctx(w)
    ctx.set_warps_per_target(wpt)
    J, F = evaluate(ctx)
    Jr, Fr = orc.Tree(w).evaluate()
    assert np.abs(J / Jr - 1).max() <= 1e-4
    assert flux_err(F, Fr, Jr).max() <= 1e-4


def test_autotune_picks_a_team_size(orc):
    w = synth.turbulent_cloud(32)
    ctx, _ = build_ctx(w)
    best, ms = ctx.autotune(8192)
    assert best in (2, 3, 4, 8) and all(m > 0 for m in ms)  # no thick material: all four tried
    assert ms[(2, 3, 4, 8).index(best)] == min(ms)
    J, F = evaluate(ctx)
    tg = synth.sample_targets(w.n_leaves, 256, seed=3)
    Jr, _ = orc.Tree(w).evaluate(tg)
    assert np.abs(J[tg] / Jr - 1).max() <= 1e-4


def test_batch_larger_than_one_launch(orc):
    """More boxes than one launch's parameters hold (97): the batch runs in chunks; every
    box matches its own single-box evaluation, thin and thick boxes mixed."""
    import torch

    import paper_2204_09072_gb300 as tr
    ws = [synth.random_uniform(8, seed=300 + k, thick_frac=0.1 if k % 3 == 0 else 0.0, n_stars=1)
          for k in range(203)]
    ctxs = [build_ctx(w)[0] for w in ws]
    singles = [evaluate(c) for c in ctxs]
    b = tr.Batch(ctxs)
    Js = [torch.empty(c.leaf_count, dtype=torch.float32, device="cuda:0") for c in ctxs]
    Fs = [torch.empty(3 * c.leaf_count, dtype=torch.float64, device="cuda:0") for c in ctxs]
    b.evaluate(Js, Fs, use_graph=True)
    for c in ctxs:
        c.check()
    for (Js1, Fs1), J, F in zip(singles, Js, Fs):
        J = J.double().cpu().numpy()
        F = F.cpu().numpy().reshape(-1, 3)
        assert np.abs(J / Js1 - 1).max() < 1e-5
        assert flux_err(F, Fs1, Js1).max() < 1e-5
    Jr, Fr = orc.Tree(ws[150]).evaluate()
    J = Js[150].double().cpu().numpy()
    assert np.abs(J / Jr - 1).max() <= 1e-4
    b.close()
    for c in ctxs:
        c.close()


def test_autotune_skips_three_warps_with_thick_material(orc):
    w = synth.random_uniform(16, seed=14, thick_frac=0.2)
    ctx, _ = build_ctx(w)
    best, ms = ctx.autotune(4096)
    assert ms[1] == -1.0 and best in (2, 4, 8)
    ctx.set_warps_per_target(3)  # runs as four on a tree with thick material
    J, F = evaluate(ctx)
    Jr, Fr = orc.Tree(w).evaluate()
    assert np.abs(J / Jr - 1).max() <= 1e-4 and flux_err(F, Fr, Jr).max() <= 1e-4
