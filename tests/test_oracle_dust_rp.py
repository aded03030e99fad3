"""Dust temperature (Sec. 4.6, App. D) and radiation-pressure (Sec. 4.5) pins."""
import math

import numpy as np

import synth

SIGMA = 5.670374419e-5
C = 2.99792458e10


def test_radiative_limit_is_radiation_temperature(orc):
    # tiny density: gas coupling negligible, T_d = T_J = (pi J / sigma)^(1/4) (eq. radtemp)
    p = synth.default_params(kappa_model=1)
    for TJ in [5.0, 20.0, 80.0, 300.0]:
        J = SIGMA * TJ ** 4 / math.pi
        td = orc.td_solve(p, 1e-30, 50.0, J)
        assert math.isclose(td, TJ, rel_tol=1e-9)


def test_floor_and_gas_limit(orc):
    p = synth.default_params(kappa_model=0, kappa0=1.0)
    assert orc.td_solve(p, 1e-22, 1.0, 0.0) == 2.7
    # very dense: dust locks to the gas temperature
    td = orc.td_solve(p, 1e-10, 35.0, SIGMA * 10.0 ** 4 / math.pi)
    assert abs(td / 35.0 - 1) < 1e-3


def test_residual_zero(orc):
    rng = np.random.default_rng(5)
    p = synth.default_params(kappa_model=1)
    rho = 10 ** rng.uniform(-22, -16, 200).astype(np.float32)
    tg = rng.uniform(5, 200, 200).astype(np.float32)
    J = SIGMA * rng.uniform(3, 60, 200) ** 4 / math.pi
    heat = (rng.uniform(0, 1, 200) * 1e-24).astype(np.float32)
    td = orc.dust_temperature(p, rho, tg, J, heat)
    for k in range(200):
        T = td[k]
        kap = 1e-3 * min(T, 150.0) ** 2
        nH = 0.7 * float(rho[k]) / 1.6726e-24
        gd = 3.8e-33 * math.sqrt(tg[k]) * (tg[k] - T) * (1 - 0.8 * math.exp(-75 / tg[k])) * nH * nH
        rad = float(rho[k]) * kap * (4 * math.pi * J[k] + 0 - 4 * SIGMA * T ** 4)
        scale = abs(gd) + float(heat[k]) + float(rho[k]) * kap * 4 * math.pi * J[k] + 1e-300
        if T > 2.7:
            assert abs(gd + float(heat[k]) + rad) <= 1e-6 * scale


def test_radpressure_limits(orc):
    # thin cell: a = kappa F / c; thick cell: force -> F dx^2 / c
    w = synth.point_source(8, kappa0=1.0)
    t = orc.Tree(w)
    J, F = t.evaluate()
    u, a, f, ps = t.radpressure(J, F)
    assert np.allclose(u, 4 * math.pi * J / C, rtol=1e-14)
    lv = t.leaves()
    g = (1 - np.exp(-lv["tau"])) / lv["tau"]
    assert np.allclose(a, F * (lv["kappa"] * g)[:, None] / C, rtol=1e-12)
    assert (ps[lv["jsrc"] > 0] > 0).all()
    w2 = synth.point_source(8, kappa0=1.0, rho0=1e-13)  # tau_cell ~ 1e3
    t2 = orc.Tree(w2)
    J2, F2 = t2.evaluate()
    u2, a2, f2, _ = t2.radpressure(J2, F2)
    dx = w2.box_cm / 8
    assert np.allclose(f2, F2 * dx * dx / C, rtol=2e-3)


def test_uv_radpressure_stroemgren_balance(orc):
    """UV radiation pressure (App. C) tied to the Stroemgren sphere of the HII-region test
    (eq. stroemgren, alpha_B = 2.5e-13 cm^3/s): inside a fully ionised uniform sphere of
    radius R_s = (3 N / (4 pi alpha_B n^2))^(1/3) around a source of N ionising photons/s,
    recombinations balance the source, so the recombination term summed over the sphere
    carries the photon momentum N E / c (E = 18 eV) whatever the grid; the force points
    along the photon direction, and a fully neutral cell feels only the absorption terms."""
    import math
    n = 32
    w = synth.homogeneous(n, 1.0, 1e-21)  # n_H = 0.7 rho / m_H ~ 0.42 cm^-3
    t = orc.Tree(w)
    nh = 0.7 * float(w.rho[0]) / 1.6726e-24  # the FP32 density the tree holds
    Rs = 0.35 * w.box_cm
    N = 4 * math.pi / 3 * Rs ** 3 * 2.5e-13 * nh * nh
    cen = synth.cell_centres(n, w.box_cm)
    r = cen - 0.5 * w.box_cm
    d = np.linalg.norm(r, axis=1)
    u = r / d[:, None]
    inside = d < Rs
    x = np.where(inside, 1.0, 0.0)
    a, f = t.uv_radpressure(np.zeros(n ** 3), u, x)  # no flux: recombination term only
    p_tot = np.linalg.norm(f[inside], axis=1).sum()
    E = 18.0 * 1.602176634e-12
    assert abs(p_tot / (N * E / 2.99792458e10) - 1) < 0.02  # the sphere on a 32^3 grid
    assert np.allclose(np.cross(f, u), 0.0, atol=1e-12 * np.abs(f).max())
    assert np.allclose(a * (w.rho.astype(np.float64)[:, None] * (w.box_cm / n) ** 3), f, rtol=1e-12)
    # a neutral cell under a photon flux: dust and neutral-H absorption, sigma_d + sigma_H
    nph = np.full(n ** 3, 1e8)
    a0, f0 = t.uv_radpressure(nph, u, np.zeros(n ** 3))
    expect = (1.5e-21 + 6.3e-18) * nh * 1e8 * E / 2.99792458e10 * (w.box_cm / n) ** 3
    assert np.allclose(np.linalg.norm(f0, axis=1), expect, rtol=1e-12)
