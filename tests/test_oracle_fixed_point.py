"""Pins of the oracle's dust-temperature / IR-field fixed point (Sec. 4.6)."""
import numpy as np

import synth


def test_gas_locked_limit(orc):
    """Dense gas couples the dust to the gas: the fixed point sits at T_gas."""
    w = synth.homogeneous(8, 0.01, 1e-12, td=10.0, kappa0=0.01)
    tgas = np.full(w.n_leaves, 35.0, np.float32)
    td, it, hist = orc.fixed_point(w, tgas, w.td, max_iter=50, tol=1e-5)
    assert it > 0
    assert np.allclose(td, 35.0, rtol=2e-3)


def test_fixed_point_is_self_consistent(orc):
    """At convergence the balance with the J of the converged T_d reproduces T_d."""
    w = synth.with_gas(synth.turbulent_cloud(16, seed=5), seed=7)
    td, it, hist = orc.fixed_point(w, w.tgas, w.td, max_iter=60, tol=1e-6)
    assert it > 0 and hist[-1] < 1e-6
    w.td = td
    J, _ = orc.Tree(w).evaluate()
    tn = orc.dust_temperature(w.params, w.rho, w.tgas, J)
    assert np.abs(tn / td - 1).max() < 1e-5
    # contraction: the changes shrink once the iteration settles
    assert hist[-1] < hist[1]


def test_weak_coupling_cools_to_floor(orc):
    """Thin, tenuous gas without sources: dust radiates its heat away toward 2.7 K."""
    w = synth.homogeneous(8, 1.0, 1e-24, td=20.0, kappa0=1.0)
    tgas = np.full(w.n_leaves, 2.0, np.float32)
    td, it, _ = orc.fixed_point(w, tgas, w.td, max_iter=50, tol=1e-5)
    assert it > 0
    assert np.allclose(td, 2.7, rtol=1e-6)


def test_thick_cells_under_outside_heating_do_not_settle(orc):
    """The own segment of a target has no optical depth (eqs. tauthin and opt thick at
    i = 0), so a thick cell's own emission gives it J = sigma T^4 / pi (App. B) while all
    outside radiation still arrives: its radiative cooling is cancelled and only the
    weak gas coupling can balance the heating. The same box with thin dust settles in a
    few iterations; with thick dust the iteration keeps heating."""
    runs = {}
    for kappa0 in (10.0, 0.1):  # tau_b ~ 3 and ~ 0.03 per cell
        w = synth.point_source(8, box_pc=0.1, rho0=7.7e-18, kappa0=kappa0, lum_lsun=1e3)
        w.params = dict(w.params, dust_emission=1)
        tgas = np.full(w.n_leaves, 20.0, np.float32)
        td0 = np.full(w.n_leaves, 20.0, np.float32)
        runs[kappa0] = orc.fixed_point(w, tgas, td0, max_iter=40, tol=1e-4)
    td, it, hist = runs[0.1]
    assert 0 < it <= 10
    td, it, hist = runs[10.0]
    assert it < 0  # not converged after 40 iterations
    assert min(hist[-10:]) > 1e-3
