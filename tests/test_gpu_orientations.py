"""Several HEALPix orientations (Sec. 7.6) on the GPU against the FP64 oracle, through the
C ABI: each target uses the angular kernel and ray directions of its own orientation.
J within 1e-4 relative, F within 1e-4 of max(|F|, 1e-2 x 4 pi J); walk totals exact."""
import numpy as np
import pytest

import synth
from gpu_util import build_ctx, evaluate, flux_err

pytestmark = pytest.mark.gpu

J_TOL = 1e-4
F_TOL = 1e-4


def _map(n, k, seed):
    return np.random.Generator(np.random.PCG64(seed)).integers(0, k, n).astype(np.uint8)


# (workload, number of orientations, rotation seed, map seed or None for leaf mod k)
CASES = {
    "rand16_k4": (lambda: synth.random_uniform(16, seed=10, thick_frac=0.15, n_stars=3), 4, 41, None),
    "clump16_k3_map": (lambda: synth.gaussian_clump(16), 3, 42, 5),
    "rand16_192_k2": (lambda: synth.random_uniform(16, seed=11, thick_frac=0.1, npix=192, nbins=16), 2, 43, 6),
    # closest periodic copies (ties split in two) and mapping at the COL: the general kernel
    "amr_periodic_col_k5": (lambda: synth.amr_core(n_base_blocks=2, max_level=2, target_leaves=24 * 512,
                                                   n_stars=3, periodic=1, col_mapping=1), 5, 44, 7),
    "rand16_periodic_k8": (lambda: synth.random_uniform(16, seed=12, thick_frac=0.1, n_stars=2, periodic=7),
                           8, 45, None),
}


def _setup(orc, name):
    import torch
    make, k, rseed, mseed = CASES[name]
    w = make()
    R = synth.random_rotations(k, seed=rseed)
    m = None if mseed is None else _map(w.n_leaves, k, mseed)
    t = orc.Tree(w)
    t.set_orientations(R, m)
    ctx, _ = build_ctx(w)
    ctx.set_orientations(R, None if m is None else torch.as_tensor(m, device="cuda:0"))
    return w, t, ctx


@pytest.mark.parametrize("name", list(CASES))
def test_evaluate_turned_rays(orc, name):
    w, t, ctx = _setup(orc, name)
    Jr, Fr = t.evaluate()
    J, F = evaluate(ctx)
    ej = np.abs(J / Jr - 1)
    ef = flux_err(F, Fr, Jr)
    assert ej.max() <= J_TOL, (ej.max(), np.argmax(ej))
    assert ef.max() <= F_TOL, (ef.max(), np.argmax(ef))
    tg = synth.sample_targets(w.n_leaves, 333, seed=4)  # ragged subset through a target list
    J, F = evaluate(ctx, tg)
    Jr, Fr = t.evaluate(tg)
    assert np.abs(J / Jr - 1).max() <= J_TOL and flux_err(F, Fr, Jr).max() <= F_TOL


@pytest.mark.parametrize("name", list(CASES))
def test_walk_stats_turned_rays(orc, name):
    import torch
    w, t, ctx = _setup(orc, name)
    tg = synth.sample_targets(w.n_leaves, 200, seed=8)
    ref = np.array([t.walk_stats(int(k)) for k in tg]).sum(0)
    got = ctx.walk_stats(torch.as_tensor(tg, dtype=torch.int32, device="cuda:0")).cpu().numpy()
    assert (got == ref).all(), (got, ref)


def test_orientations_before_build_and_reset(orc):
    """Set before the first build: the tables follow at the build, with leaf mod k. k = 0
    goes back to the single unturned ray set."""
    import paper_2204_09072_gb300 as tr
    w = synth.random_uniform(16, seed=13, thick_frac=0.1)
    R = synth.random_rotations(3, seed=46)
    t = orc.Tree(w)
    t.set_orientations(R)
    Jr, Fr = t.evaluate()
    ctx = tr.Context(w.params)
    ctx.set_orientations(R)
    import torch
    dev = torch.device("cuda:0")
    ctx.build(w.box_cm, torch.from_numpy(w.rho).to(dev), torch.from_numpy(w.td).to(dev), n=w.uniform_n,
              star_pos=w.star_pos, star_lum=w.star_lum)
    J, F = evaluate(ctx)
    assert np.abs(J / Jr - 1).max() <= J_TOL and flux_err(F, Fr, Jr).max() <= F_TOL
    ctx.set_orientations(np.zeros((0, 3, 3)))
    J, F = evaluate(ctx)
    Jr, Fr = orc.Tree(w).evaluate()
    assert np.abs(J / Jr - 1).max() <= J_TOL and flux_err(F, Fr, Jr).max() <= F_TOL


def test_batch_with_turned_rays(orc):
    """Two boxes in one persistent launch, each with its own orientations."""
    import torch

    import paper_2204_09072_gb300 as tr
    ws = [synth.random_uniform(16, seed=14, thick_frac=0.1), synth.gaussian_clump(16)]
    ctxs, refs = [], []
    for i, w in enumerate(ws):
        R = synth.random_rotations(2 + i, seed=47 + i)
        t = orc.Tree(w)
        t.set_orientations(R)
        refs.append(t.evaluate())
        c, _ = build_ctx(w)
        c.set_orientations(R)
        ctxs.append(c)
    b = tr.Batch(ctxs)
    Js = [torch.empty(w.n_leaves, dtype=torch.float32, device="cuda:0") for w in ws]
    Fs = [torch.empty(3 * w.n_leaves, dtype=torch.float64, device="cuda:0") for w in ws]
    b.evaluate(Js, Fs, use_graph=False)
    for c in ctxs:
        c.check()
    for (Jr, Fr), J, F in zip(refs, Js, Fs):
        J = J.cpu().numpy().astype(np.float64)
        F = F.cpu().numpy().reshape(-1, 3)
        assert np.abs(J / Jr - 1).max() <= J_TOL and flux_err(F, Fr, Jr).max() <= F_TOL
    b.close()


def test_orientation_errors():
    import torch

    import paper_2204_09072_gb300 as tr
    w = synth.gaussian_clump(8)
    ctx = tr.Context(w.params)
    with pytest.raises(tr.TreeRayError) as e:  # a map needs a built tree
        ctx.set_orientations(np.eye(3)[None], torch.zeros(512, dtype=torch.uint8, device="cuda:0"))
    assert e.value.code == 4
    ctx, _ = build_ctx(w)
    with pytest.raises(tr.TreeRayError) as e:
        ctx.set_orientations(2.0 * np.eye(3)[None])
    assert e.value.code == 1
    with pytest.raises(tr.TreeRayError) as e:
        ctx.set_orientations(np.eye(3)[None], torch.ones(512, dtype=torch.uint8, device="cuda:0"))
    assert e.value.code == 1
    with pytest.raises(tr.TreeRayError) as e:
        ctx.set_orientations(np.tile(np.eye(3), (65, 1, 1)))
    assert e.value.code == 1
