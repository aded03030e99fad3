"""The optically thick blob test (Sec. 5.2, optically thick blob of dust) as pins of the
oracle's thick path: blobs S, M, L (0.75, 1.5, 3 pc across) at 30 K in a (15 pc)^3 box,
with ambient gas at 10 K (S, M, L), without it (S-, M-, L-) or ten times denser (S+),
on 64^3 cells (S is 2 x 2 x 2 cells, as in the paper's runs)."""
import math

import numpy as np
import pytest

import synth

SIGMA = 5.670374419e-5
PC = 3.0857e18
N = 64


@pytest.fixture(scope="module")
def geom():
    w = synth.blob_suite("S", N)
    cen = synth.cell_centres(N, w.box_cm) - 0.5 * w.box_cm
    r = np.sqrt((cen ** 2).sum(1))
    tg = np.sort(np.random.Generator(np.random.PCG64(0)).choice(N ** 3, 6000, replace=False))
    return dict(cen=cen, r=r, tg=tg, dx=w.box_cm / N)


def _run(orc, variant, g):
    w = synth.blob_suite(variant, N)
    J, F = orc.Tree(w).evaluate(g["tg"])
    core = w.rho > 5e-18
    return w, J, F, core


def _far_unit(core, dx):
    """J r^2 of the whole blob seen as one thick node through one ray: the node's solid
    angle is (Q/V) V^(2/3) / R_i^2 = V^(2/3) / r^2 (beta = R_i^2 / r^2) and its intensity
    sigma T^4 / pi, so J = sigma T^4 V^(2/3) / (4 pi^2 r^2) (eqs. omegaThick, opt thick)."""
    V = core.sum() * dx ** 3
    return SIGMA * 30.0 ** 4 * V ** (2.0 / 3.0) / (4 * math.pi ** 2)


def test_far_field_scales_with_the_cross_section(orc, geom):
    """Without ambient gas the far field of the blob follows the inverse square law and
    scales with the blob's cross-section V^(2/3) (not its volume): J r^2 over the shell
    4.5-7 pc, in units of the one-node-one-ray value, is the same for S-, M- and L- within
    3 %, and lies between that value (1) and a split of the blob into its eight octants,
    each spread over up to three rays (8^(1/3) x 1.44). The shell averages at 4.5-5.5 and
    6-7 pc agree within 3 % (r^-2)."""
    tg, r = geom["tg"], geom["r"][geom["tg"]]
    shell = (r > 4.5 * PC) & (r < 7.0 * PC)
    inner = (r > 4.5 * PC) & (r < 5.5 * PC)
    outer = (r > 6.0 * PC) & (r < 7.0 * PC)
    vals = {}
    for v in ("S-", "M-", "L-"):
        w, J, F, core = _run(orc, v, geom)
        x = J * r ** 2 / _far_unit(core, geom["dx"])
        vals[v] = x[shell].mean()
        assert 1.0 <= x[shell].min() and x[shell].max() <= 2.0 * 1.44, (v, x[shell].min(), x[shell].max())
        assert abs(x[inner].mean() / x[outer].mean() - 1) < 0.03, v
    for v in ("M-", "L-"):
        assert abs(vals[v] / vals["S-"] - 1) < 0.03, vals


def test_far_field_flux_points_away_from_the_blob(orc, geom):
    w, J, F, core = _run(orc, "S-", geom)
    c = geom["cen"][geom["tg"]]
    r = np.linalg.norm(c, axis=1)
    far = r > 2.0 * PC
    radial = (F[far] * c[far]).sum(1) / r[far] / (4 * math.pi * J[far])
    assert radial.min() > 0.85
    assert (np.linalg.norm(F[far], axis=1) <= 4 * math.pi * J[far] * (1 + 1e-12)).all()


@pytest.mark.parametrize("variant", ["M", "L"])
def test_plateau_inside_the_blob(orc, geom, variant):
    """Deep inside an isothermal thick body every ray ends on material at T_c:
    J = sigma T_c^4 / pi (App. B) and, by symmetry, F = 0."""
    w = synth.blob_suite(variant, N)
    R = 0.5 * synth.BLOB_DIAMETER_PC[variant] * PC
    inside = np.nonzero(geom["r"] < R - 1.5 * geom["dx"])[0]  # every interior cell
    assert len(inside) >= 8
    J, F = orc.Tree(w).evaluate(inside)
    J30 = SIGMA * 30.0 ** 4 / math.pi
    assert np.abs(J / J30 - 1).max() < 0.01
    assert (np.linalg.norm(F, axis=1) < 1e-3 * 4 * math.pi * J).all()


def test_dense_ambient_tends_to_its_own_temperature(orc, geom):
    """S+: the ambient gas is optically thick across the box, so where the blob's light
    has faded J approaches the 10 K value sigma T_a^4 / pi from below (the box has no
    background radiation)."""
    w, J, F, core = _run(orc, "S+", geom)
    r = geom["r"][geom["tg"]]
    mid = (r > 3.5 * PC) & (r < 5.5 * PC)
    x = J[mid] / (SIGMA * 10.0 ** 4 / math.pi)
    assert 0.85 < x.min() and x.max() < 1.0
    # the thinner ambient of S stays well below it
    w, J, F, core = _run(orc, "S", geom)
    assert (J[mid] / (SIGMA * 10.0 ** 4 / math.pi)).max() < 0.5


def _rect_solid_angle(x1, x2, y1, y2, z):
    """Solid angle of the rectangle [x1, x2] x [y1, y2] in a plane at distance z > 0,
    seen from the origin (sum of the corner terms atan(x y / (z sqrt(x^2 + y^2 + z^2))))."""
    def f(x, y):
        return math.atan(x * y / (z * math.sqrt(x * x + y * y + z * z)))
    return f(x2, y2) - f(x1, y2) - f(x2, y1) + f(x1, y1)


def _box_solid_angle(p, lo, hi):
    """Exact solid angle of an axis-aligned box seen from an outside point: its faces that
    face the point."""
    om = 0.0
    for a in range(3):
        b, c = [k for k in range(3) if k != a]
        for plane, facing in ((lo[a], p[a] < lo[a]), (hi[a], p[a] > hi[a])):
            if facing:
                om += _rect_solid_angle(lo[b] - p[b], hi[b] - p[b], lo[c] - p[c], hi[c] - p[c],
                                        abs(plane - p[a]))
    return om


def test_far_field_against_the_exact_opaque_box(orc, geom):
    """S- on 64^3 is a 2 x 2 x 2 block of cells with tau_b = 13 each, i.e. an opaque box:
    a target outside sees B = sigma T^4 / pi over the box's solid angle Omega, so exactly
    J = B Omega / (4 pi). The method sees the blob through nodes mapped onto rays: one
    thick node in one ray gives V^(2/3) / r^2, between 1/sqrt(3) of the projected area
    (corner on) and all of it (face on); the eight octants split over up to three rays
    each raise it to at most 8^(1/3) x 1.44 times that (the thick-mapping overestimate of
    Sec. 7.6). Per target the ratio to the exact J stays within those bounds, and its mean
    over every shell is an overestimate of less than 30 %."""
    w, J, F, core = _run(orc, "S-", geom)
    cen = synth.cell_centres(N, w.box_cm)
    dx = geom["dx"]
    lo = cen[core].min(0) - 0.5 * dx
    hi = cen[core].max(0) + 0.5 * dx
    assert np.allclose((hi - lo) / dx, 2.0)
    tg, r = geom["tg"], geom["r"][geom["tg"]]
    far = r > 1.0 * PC
    B = SIGMA * 30.0 ** 4 / math.pi
    exact = np.array([B * _box_solid_angle(cen[k], lo, hi) / (4 * math.pi) for k in tg[far]])
    ratio = J[far] / exact
    assert ratio.min() >= 1.0 / math.sqrt(3.0) and ratio.max() <= 2.0 * 1.44
    for a, b in ((1.0, 3.0), (3.0, 5.0), (5.0, 7.5)):
        m = (r[far] > a * PC) & (r[far] < b * PC)
        assert 1.0 <= ratio[m].mean() <= 1.3, (a, b, ratio[m].mean())
