"""HEALPix pins for the oracle (nested scheme, Gorski et al. 2005).

Textbook facts: base-pixel centres at z = 2/3, 0, -2/3 and phi = pi/4 + k pi/2
(north/south) or k pi/2 (equator); every pixel centre maps back to its own
pixel; equal areas; antipodal symmetry; nested children lie in their parent.
"""
import math

import numpy as np
import pytest


def test_base_pixel_centres(orc):
    for p in range(12):
        v = orc.pix2vec(1, p)
        row, k = divmod(p, 4)
        z_expect = [2.0 / 3.0, 0.0, -2.0 / 3.0][row]
        phi_expect = (k * math.pi / 2 + (0.0 if row == 1 else math.pi / 4))
        assert abs(v[2] - z_expect) < 1e-14
        phi = math.atan2(v[1], v[0]) % (2 * math.pi)
        assert abs(phi - phi_expect) < 1e-12
        assert abs(np.linalg.norm(v) - 1) < 1e-14


@pytest.mark.parametrize("nside", [1, 2, 4, 8])
def test_roundtrip_and_symmetry(orc, nside):
    npix = 12 * nside * nside
    vecs = np.array([orc.pix2vec(nside, p) for p in range(npix)])
    for p in range(npix):
        assert orc.ang2pix(nside, vecs[p]) == p
    assert np.abs(vecs.sum(0)).max() < 1e-12
    # antipode of every centre is a centre
    for p in range(npix):
        q = orc.ang2pix(nside, -vecs[p])
        assert np.allclose(vecs[q], -vecs[p], atol=1e-12)


def test_nested_children_in_parent(orc):
    for p in range(48):
        assert orc.ang2pix(1, orc.pix2vec(2, p)) == p // 4
    for p in range(192):
        assert orc.ang2pix(2, orc.pix2vec(4, p)) == p // 4


@pytest.mark.parametrize("nside", [2, 4])
def test_equal_area(orc, nside):
    npix = 12 * nside * nside
    n = 120000
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    phi = math.pi * (1 + 5 ** 0.5) * i
    s = np.sqrt(1 - z * z)
    counts = np.zeros(npix)
    for k in range(n):
        counts[orc.ang2pix(nside, (s[k] * math.cos(phi[k]), s[k] * math.sin(phi[k]), z[k]))] += 1
    # Fibonacci directions: discretisation noise of a few per cent per pixel
    assert np.abs(counts / (n / npix) - 1).max() < 0.05
    assert np.abs(counts / (n / npix) - 1).mean() < 0.015
