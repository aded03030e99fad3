"""Pins of the oracle's several HEALPix orientations (Sec. 7.6): a turned ray set is the
HEALPix grid rotated by R, so a direction v belongs to ray h when R^T v lies in pixel h,
and ray h points along R n^h. Checked against what geometry fixes: the identity, the
quarter turn about the polar axis (a symmetry of the HEALPix grid), the orientation
independence of J without extinction, and the direction of the flux from a point source."""
import math

import numpy as np
import pytest

import synth

RZ90 = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])  # +90 deg about z
RX90 = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])  # +90 deg about x

KEYS = [(8, 0, 0), (16, 8, -8), (3, 5, -7), (24, -16, 40), (1, 1, 1), (-9, 7, 3), (0, 0, -24),
        (-40, 13, 21), (2, -6, 10), (5, 5, 5), (-4, 12, -20), (33, -31, 1)]


def _perm(orc, nside, R):
    """pi(h): the pixel whose centre is R n^h (R a symmetry of the grid)."""
    npix = 12 * nside * nside
    n = np.array([orc.pix2vec(nside, h) for h in range(npix)])
    rn = n @ R.T
    d = np.linalg.norm(rn[:, None, :] - n[None, :, :], axis=2)
    p = d.argmin(1)
    assert d[np.arange(npix), p].max() < 1e-12
    return p


@pytest.mark.parametrize("npix", [12, 48, 192])
def test_quarter_turn_permutes_the_rays(orc, npix):
    """The quarter turn about z maps every HEALPix pixel onto another one, so the rays of
    the turned set are the pixels pi(h) with centre R n^h and the hit counts are permuted:
    counts_R(K)[h] = counts(K)[pi(h)]. With R^T in place of R the permutation is the
    inverse one, which the keys below tell apart."""
    nside = int(round(math.sqrt(npix / 12)))
    p = _perm(orc, nside, RZ90)
    pinv = np.argsort(p)
    differs = False
    for K in KEYS:
        c0 = orc.alpha_counts(npix, K)
        cr = orc.alpha_counts(npix, K, rot=RZ90)
        assert np.array_equal(cr, c0[p]), K
        assert cr.sum() == 512
        differs |= not np.array_equal(cr, c0[pinv])
    assert differs


def test_identity_rotation_is_the_unturned_grid(orc):
    w = synth.random_uniform(8, seed=4)
    t = orc.Tree(w)
    J0, F0 = t.evaluate()
    s0 = [t.walk_stats(k) for k in (0, 100, 511)]
    t.set_orientations(np.eye(3)[None])
    J1, F1 = t.evaluate()
    assert np.array_equal(J0, J1) and np.array_equal(F0, F1)
    assert all(np.array_equal(a, t.walk_stats(k)) for a, k in zip(s0, (0, 100, 511)))
    t.set_orientations(np.zeros((0, 3, 3)))  # back to the single unturned set
    J2, F2 = t.evaluate()
    assert np.array_equal(J0, J2) and np.array_equal(F0, F2)


def test_quarter_turn_leaves_the_field_unchanged(orc):
    """Turning the rays by a symmetry of the grid changes only the order of the rays:
    J and F (thin and thick material, straddle merges, extinction) equal the unturned
    ones up to rounding. Inconsistent use of R (R^T for the mapping, R for the
    directions, or the reverse) would turn F by 180 degrees about z."""
    w = synth.random_uniform(8, seed=5)
    t = orc.Tree(w)
    J0, F0 = t.evaluate()
    t.set_orientations(RZ90[None])
    J1, F1 = t.evaluate()
    assert np.allclose(J1, J0, rtol=1e-12, atol=0)
    scale = np.linalg.norm(F0, axis=1, keepdims=True)
    assert np.abs(F1 - F0).max() / scale.max() < 1e-12
    assert (np.abs(F1 - F0) <= 1e-11 * scale + 1e-300).all()


def test_thin_J_independent_of_orientation(orc):
    """Without extinction J = sum_i sum_h L^_ih / (16 pi^2 R_i^2) and sum_h alpha_h = 1
    for every orientation, so J does not depend on the rays' orientation."""
    w = synth.random_uniform(8, seed=3, thick_frac=0.0, kappa_ext_scale=0.0)
    t = orc.Tree(w)
    J0, F0 = t.evaluate()
    R = synth.random_rotations(5, seed=21)
    orient = np.random.Generator(np.random.PCG64(9)).integers(0, 5, w.n_leaves).astype(np.uint8)
    t.set_orientations(R, orient)
    J1, F1 = t.evaluate()
    assert np.allclose(J1, J0, rtol=1e-12, atol=0)
    assert not np.allclose(F1, F0, rtol=1e-6)  # the flux directions do change


def test_orientation_map_selects_each_targets_rays(orc):
    """A target with orientation o gets exactly the result of a single-orientation run
    with R_o; the default map is leaf mod k."""
    w = synth.random_uniform(8, seed=6)
    t = orc.Tree(w)
    R = synth.random_rotations(3, seed=22)
    single = []
    for o in range(3):
        t.set_orientations(R[o:o + 1])
        single.append(t.evaluate())
    orient = np.random.Generator(np.random.PCG64(2)).integers(0, 3, w.n_leaves).astype(np.uint8)
    t.set_orientations(R, orient)
    J, F = t.evaluate()
    for o in range(3):
        m = orient == o
        assert np.array_equal(J[m], single[o][0][m]) and np.array_equal(F[m], single[o][1][m])
    t.set_orientations(R)
    J, F = t.evaluate()
    mod = np.arange(w.n_leaves) % 3
    for o in range(3):
        m = mod == o
        assert np.array_equal(J[m], single[o][0][m]) and np.array_equal(F[m], single[o][1][m])


@pytest.mark.parametrize("rot", ["x90", "random"])
def test_turned_rays_point_the_flux_away_from_a_point_source(orc, rot):
    """A lone point source without extinction: each far target's flux is a mix of the
    turned ray directions R n^h of the pixels the source falls into, so it points away
    from the source to within the largest pixel radius plus the source cell's angular
    radius. (R^T for the mapping and R for the directions would put it well off.)"""
    n = 16
    R = RX90 if rot == "x90" else synth.random_rotations(1, seed=23)[0]
    w = synth.point_source(n, kappa0=0.0, cell=(3, 4, 5))
    t = orc.Tree(w)
    t.set_orientations(R[None])
    cen = synth.cell_centres(n, w.box_cm)
    src = w.star_pos[0]
    dist = np.linalg.norm(cen - src, axis=1)
    tg = np.nonzero(dist > 6.0 * w.box_cm / n)[0]
    _, F = t.evaluate(tg)
    true = (cen[tg] - src) / dist[tg, None]
    ang = np.arccos(np.clip((F * true).sum(1) / np.linalg.norm(F, axis=1), -1, 1))
    # largest angle between a direction and the centre of its pixel (nside 2), sampled
    g = np.random.Generator(np.random.PCG64(1)).normal(size=(20000, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    cpix = np.array([orc.pix2vec(2, orc.ang2pix(2, v)) for v in g])
    rho_max = np.arccos(np.clip((g * cpix).sum(1), -1, 1)).max()
    cell = math.atan(math.sqrt(3) * 0.5 / 6.0)
    assert ang.max() < rho_max * 1.02 + cell
    assert np.degrees(ang.mean()) < 12.0


def test_bad_orientations_are_refused(orc):
    t = orc.Tree(synth.random_uniform(8, seed=4))
    with pytest.raises(ValueError):
        t.set_orientations((2.0 * np.eye(3))[None])  # not orthonormal
    with pytest.raises(ValueError):
        t.set_orientations(np.diag([1.0, 1.0, -1.0])[None])  # a reflection
    with pytest.raises(ValueError):
        t.set_orientations(np.eye(3)[None], np.full(512, 1, np.uint8))  # map value >= k
