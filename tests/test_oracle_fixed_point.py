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
