"""Degenerate inputs against the FP64 oracle, through the C ABI (marked gpu): a grid of one
cell (the root is a leaf) and of 2^3 cells, an empty target list, a single radial
segment, the smallest and largest opening angles, a box that is thick everywhere, and
stars outside the box (their host is the nearest edge cell on both sides), and a target
list longer than the grid."""
import numpy as np
import pytest

import synth
from gpu_util import build_ctx, evaluate, flux_err

pytestmark = pytest.mark.gpu


def _check(orc, w, targets=None):
    t = orc.Tree(w)
    ctx, _ = build_ctx(w)
    o, g = t.leaves(), ctx.leaf_export()
    for k in ("kappa", "tau", "thick"):
        assert (g[k] == o[k]).all(), k
    for k in ("jsrc", "psrc"):
        assert np.allclose(g[k], o[k], rtol=1e-14, atol=0), k
    oe, ge = t.export(), ctx.tree_export()
    for k in ("level", "leaf", "child0", "centre"):
        assert (ge[k] == oe[k]).all(), k
    J, F = evaluate(ctx, targets)
    Jr, Fr = t.evaluate(targets)
    assert np.abs(J / Jr - 1).max() <= 1e-4, np.abs(J / Jr - 1).max()
    assert flux_err(F, Fr, Jr).max() <= 1e-4
    return ctx, J, F


def test_single_cell_grid(orc):
    """One cell: the root is the only leaf, the walk has nothing to visit and J is the
    cell's own emission and star; the own cell's rays are uniform, so F is ~0."""
    w = synth.random_uniform(1, seed=3, n_stars=1)
    ctx, J, F = _check(orc, w)
    assert ctx.node_count == 1
    assert np.linalg.norm(F) <= 1e-6 * 4 * np.pi * J[0]


def test_two_by_two_by_two_grid(orc):
    _check(orc, synth.random_uniform(2, seed=4, n_stars=1))


def test_empty_target_list():
    import torch
    w = synth.random_uniform(8, seed=5)
    ctx, _ = build_ctx(w)
    J = torch.full((4,), -1.0, dtype=torch.float32, device="cuda:0")
    F = torch.full((12,), -1.0, dtype=torch.float64, device="cuda:0")
    ctx.evaluate(J, F, targets=torch.zeros(0, dtype=torch.int32, device="cuda:0"))
    ctx.check()
    assert (J == -1.0).all() and (F == -1.0).all()


def test_single_radial_segment(orc):
    _check(orc, synth.random_uniform(16, seed=6, nbins=1, thick_frac=0.15))


@pytest.mark.parametrize("theta", [1e-3, 2.0])
def test_extreme_opening_angles(orc, theta):
    """theta -> 0 accepts every leaf; theta = 2 (the largest allowed) accepts nodes as
    large as twice their distance."""
    w = synth.random_uniform(8 if theta < 0.1 else 16, seed=7, thick_frac=0.1, theta=theta)
    ctx, J, F = _check(orc, w)
    import torch
    tg = synth.sample_targets(w.n_leaves, 97, seed=2)
    ref = np.array([orc.Tree(w).walk_stats(int(k)) for k in tg]).sum(0)
    got = ctx.walk_stats(torch.as_tensor(tg, dtype=torch.int32, device="cuda:0")).cpu().numpy()
    assert (got == ref).all()


def test_thick_everywhere(orc):
    """Every cell optically thick (tau_b = 19): the thick kernel on a box without any thin
    material."""
    w = synth.homogeneous(16, 1.0, 1e-19, td=20.0, kappa_model=0, kappa0=1000.0)
    ctx, J, F = _check(orc, w)
    assert ctx.leaf_export()["thick"].all()


def test_stars_outside_the_box(orc):
    w = synth.random_uniform(8, seed=8, n_stars=3)
    w.star_pos = np.array([[-0.1, 0.5, 0.5], [0.3, 1.2, 0.9], [0.5, 0.5, 1.0]]) * w.box_cm
    _check(orc, w)


@pytest.mark.parametrize("thick_frac", [0.0, 0.15])
def test_target_list_longer_than_the_grid(orc, thick_frac):
    """A target list with repeats, three times the leaf count plus a ragged tail: more
    teams than the build reserved tiles for (up to one per leaf), so the evaluation grows
    the teams' global scratch first; every row equals the single evaluation of its leaf
    and the oracle's value."""
    w = synth.random_uniform(8, seed=17, thick_frac=thick_frac, n_stars=2)
    n = w.n_leaves
    rng = np.random.Generator(np.random.PCG64(18))
    targets = np.concatenate([np.arange(n), rng.integers(0, n, 2 * n + 7)]).astype(np.int32)
    ctx, J1, F1 = _check(orc, w)
    J, F = evaluate(ctx, targets)
    assert np.abs(J / J1[targets] - 1).max() <= 1e-6  # FP32 reductions in any order
    assert flux_err(F, F1[targets], J1[targets]).max() <= 1e-5
    Jr, Fr = orc.Tree(w).evaluate(targets)
    assert np.abs(J / Jr - 1).max() <= 1e-4
    assert flux_err(F, Fr, Jr).max() <= 1e-4
