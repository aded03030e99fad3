"""Oracle pins against numbers evaluated by hand (outside the oracle, with 30-digit
arithmetic), each for one formula of the paper that no closed-form limit fixes:

* eq. jsrc and eq. psrc (Sec. 4.4, 4.5): the part of a star's luminosity trapped in its
  host cell, J_src = (1 - e^(-tau_b/2)) L / dx^2 and P_src = J_src / c, and the escaping
  part S = L e^(-tau_b/2) that enters the host leaf's thin luminosity (Sec. 4.1.1);
* the Planck-mean opacity law of Sec. 2, 0.1 (T / 10 K)^2 cm^2/g capped at 150 K;
* the gas-dust coupling of App. D with the Hollenbach & McKee (1989) coefficient,
  3.8e-33 sqrt(T) (T - T_d) (1 - 0.8 e^(-75/T)) n_H^2 erg/s/cm^3, n_H = 0.7 rho / m_H;
* the segment merge of Sec. 4.3 with thick content: L^_thin, A^_thin and Q^_thick scaled by
  T = R_i^2 / R_(i+1)^2, L^_thick, A^_thick and V^_thick added plainly.

Each literal below is quoted to 15+ significant digits; a wrong factor (4 pi, dx^3 for
dx^2, e^-tau for e^-tau/2, T uncapped, X = 1 for 0.7, a merged quantity scaled or not
scaled) moves the result far outside the tolerances.
"""
import math

import numpy as np

import synth

PC_CM = 3.0857e18
LSUN = 3.828e33


def test_star_source_terms_by_hand(orc):
    # 4^3 cells of (0.25 pc)^3, grey kappa 1 cm^2/g, tau_b = 0.6 in every cell; one
    # 1e4 Lsun star at the centre of cell (1, 1, 1); dust emission off
    n, dx = 4, 0.25 * PC_CM                       # dx = 7.71425e17 cm, dx^2 = 5.95096530625e35
    w = synth.point_source(n, box_pc=1.0, rho0=0.6 / dx, kappa0=1.0, lum_lsun=1e4, cell=(1, 1, 1))
    host = 1 + 4 * 1 + 16 * 1
    t = orc.Tree(w)
    lv = t.leaves()
    tau = lv["tau"][host]
    # tau_b from the float32 density differs from 0.6 by < 1e-7 relative
    assert abs(tau / 0.6 - 1) < 1e-7
    # 1 - e^-0.3 = 0.259181779318282134; L / dx^2 = 3.828e37 / 5.95096530625e35
    jsrc_hand = 16.6720489899072500      # erg/s/cm^2
    psrc_hand = 5.56119693641767664e-10  # J_src / c
    assert math.isclose(lv["jsrc"][host], jsrc_hand, rel_tol=1e-7)
    assert math.isclose(lv["psrc"][host], psrc_hand, rel_tol=1e-7)
    others = np.arange(w.n_leaves) != host
    assert (lv["jsrc"][others] == 0).all() and (lv["psrc"][others] == 0).all()
    # the escaping part S = L e^-0.3 = 2.83585214876961599e37 erg/s is the host leaf's
    # whole thin luminosity (dust emission is off)
    ex = t.export()
    node = np.nonzero(ex["leaf"] == host)[0][0]
    assert math.isclose(ex["vals"][node, 0], 2.83585214876961599e37, rel_tol=1e-7)


def test_planck_opacity_law_by_hand(orc):
    # kappa_P = 0.1 cm^2/g (T / 10 K)^2 up to 150 K, constant above (Sec. 2)
    w = synth.homogeneous(2, box_pc=1.0, rho0=1e-22, kappa_model=1)
    w.td = np.array([5.0, 20.0, 150.0, 300.0, 10.0, 40.0, 100.0, 75.0], np.float32)
    kap = orc.Tree(w).leaves()["kappa"]
    hand = [0.025, 0.4, 22.5, 22.5, 0.1, 1.6, 10.0, 5.625]
    assert np.allclose(kap, hand, rtol=1e-15, atol=0)


def test_gas_dust_coupling_by_hand(orc):
    # n_H = 1e7 cm^-3 (rho = 1e7 x 1.6726e-24 / 0.7 = 2.38942857142857143e-17 g/cm^3),
    # T_gas = 100 K, grey kappa 1 cm^2/g, J = 0. At T_d = 20 K:
    #   Gamma_dust-gas = 3.8e-33 x 10 x 80 x (1 - 0.8 e^-0.75) x 1e14
    #                  = 1.89120454373385223e-16 erg/s/cm^3
    #   cooling rho kappa 4 sigma T_d^4 = 8.67133097437202286e-16 erg/s/cm^3
    # so with the extra heating H = cooling - Gamma the balance G(T_d) = 0 sits at 20 K.
    p = synth.default_params(kappa_model=0, kappa0=1.0, dust_to_gas=0.01)
    rho = 2.38942857142857143e-17
    H = 8.67133097437202286e-16 - 1.89120454373385223e-16
    td = orc.td_solve(p, rho, 100.0, 0.0, H)
    assert math.isclose(td, 20.0, rel_tol=1e-9), td
    # the coupling scales with the dust-to-gas ratio: twice the ratio, twice Gamma
    p2 = synth.default_params(kappa_model=0, kappa0=1.0, dust_to_gas=0.02)
    H2 = 8.67133097437202286e-16 - 2 * 1.89120454373385223e-16
    assert math.isclose(orc.td_solve(p2, rho, 100.0, 0.0, H2), 20.0, rel_tol=1e-9)


def test_thick_merge_by_hand(orc):
    # four segments, R_i = 1e16 x 2^i cm, 48 rays (omega = pi / 12); the boundary between
    # segments 1 and 2 is flagged, so segment 2 folds into 1 with T = R_1^2 / R_2^2 = 1/4:
    #   L^_thin = 2e30 + 1e30 / 4 = 2.25e30      A^_thin = omega R_1^2 (0.1 + 0.3 x 4 / 4)
    #   Q^_thick = 0.8e45 + 1.8e45 / 4 = 1.25e45 L^_thick = 2e44 + 3e44 = 5e44
    #   A^_thick = 2e30 + 1e30 = 3e30            V^_thick = 1e45 + 2e45 = 3e45
    # segment 1 then has tau_thin = 0.4, omega_thick = (Q^/V^) V^^(2/3) / R_1^2
    # = 2.16675398234573345e-3, f = 8.27639056210494717e-3, tau_thick = 3.46139896873778012,
    # F*_thin = 3.68931053754397274e-4, F*_thick = 3.61125663724288909e-4, blended
    # F*_1 = 3.68926429828361029e-4; a thin source of 4e30 erg/s in segment 3 adds
    # e^-0.4 ((1 - f) + f e^-tau_thick) x 4e30 / (4 pi R_3^2)
    # = 0.664946338762032284 x 4.97359197162172924e-5.
    om = 4 * math.pi / 48
    R = 1e16 * 2.0 ** np.arange(5)
    Lth = [0, 2e30, 1e30, 4e30]
    Ath = [0, 0.1 * om * R[1] ** 2, 0.3 * om * R[2] ** 2, 1e-20]
    Lk = [0, 2e44, 3e44, 0]
    Ak = [0, 2e30, 1e30, 0]
    Vk = [0, 1e45, 2e45, 0]
    Qk = [0, 0.8e45, 1.8e45, 0]
    F = orc.ray_integrate(48, R, Lth, Ath, Lk, Ak, Vk, Qk, flag=1 << 1)
    assert math.isclose(F, 4.01998147548622093e-4, rel_tol=1e-12), F
