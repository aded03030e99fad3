"""Pins for the angular kernel alpha and its integer key (oracle)."""
import numpy as np
import pytest


def test_key_exact_cases(orc):
    # leaves (E = 2 half-units): K = 4 o exactly
    assert list(orc.alpha_key([2, -4, 0], 2)) == [8, -16, 0]
    # one level up (E = 4): K = 2 o, odd o -> K = 2 mod 4
    assert list(orc.alpha_key([3, -1, 5], 4)) == [6, -2, 10]
    # two levels up (E = 8): K = o
    assert list(orc.alpha_key([3, -1, 5], 8)) == [3, -1, 5]
    # coarser nodes: nearest odd integer to 8 o / E
    for o, E in [(1, 16), (-1, 16), (7, 16), (-7, 16), (13, 32), (-13, 32), (45, 64), (-3, 64)]:
        k = orc.alpha_key([o, 0, 0], E)[0]
        x = 8 * o / E
        assert k % 2 == 1
        assert abs(k - x) < 1.0


@pytest.mark.parametrize("K", [(1, 3, 17), (-17, 5, -3), (24, 0, 8), (-39, 39, 1), (6, -18, 2)])
def test_alpha_normalised_and_antipodal(orc, K):
    s = 8
    c = orc.alpha_counts(48, K, s)
    assert c.sum() == s ** 3
    cm = orc.alpha_counts(48, [-k for k in K], s)
    # pixel h's antipode
    anti = [orc.ang2pix(2, -orc.pix2vec(2, h)) for h in range(48)]
    for h in range(48):
        assert c[h] == cm[anti[h]]


def test_alpha_far_node_single_pixel(orc):
    # a node of edge E seen at 40 edges distance along a pixel centre falls in that pixel
    v = orc.pix2vec(2, 21)
    K = np.round(v * 8 * 40).astype(np.int64)
    c = orc.alpha_counts(48, K)
    assert c[21] == 512


def test_alpha_matches_solid_angle(orc):
    # the weights of a node spread over several pixels match the fraction of its
    # sample directions, computed here from an independent sampling of the cube
    K = (20, 4, -12)
    c = orc.alpha_counts(48, K, 8)
    rng = np.random.default_rng(0)
    pts = (np.array(K, float) / 8.0)[None, :] + rng.uniform(-0.5, 0.5, (20000, 3))
    ref = np.zeros(48)
    for p in pts:
        ref[orc.ang2pix(2, p)] += 1
    ref /= ref.sum()
    assert np.abs(c / 512.0 - ref).max() < 0.02
