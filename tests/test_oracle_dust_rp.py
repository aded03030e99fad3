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
