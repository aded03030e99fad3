"""Single-ray integration pins (Sec. 4.3 and the segment limits of App. B)."""
import math

import numpy as np

NPIX = 48
OMEGA = 4 * math.pi / NPIX


def radii(nb=4, r0=1e16):
    return r0 * 2.0 ** np.arange(nb + 1)


def test_thin_limit(orc):
    R = radii()
    L = np.array([0.0, 0.0, 3e30, 0.0])
    A = np.array([0.0, 0.0, 1e-12 * OMEGA * R[2] ** 2, 0.0])  # tau = 1e-12
    F = orc.ray_integrate(NPIX, R, L, A)
    assert math.isclose(F, 3e30 / (4 * math.pi * R[2] ** 2), rel_tol=1e-12)


def test_thick_limit_of_thin_segment(orc):
    # tau >> 1: F* -> (omega / 4 pi) L^/A^ = (4 pi / Npix)(sigma/pi) <T^4> for thin material
    R = radii()
    sigma, T = 5.670374419e-5, 30.0
    A = 1e4 * OMEGA * R[1] ** 2          # tau = 1e4
    L = 4 * sigma * T ** 4 * A           # L / A~ = 4 sigma T^4 for any node
    F = orc.ray_integrate(NPIX, R, [0, L, 0, 0], [0, A, 0, 0])
    assert math.isclose(F, 4 * math.pi / NPIX * sigma / math.pi * T ** 4, rel_tol=1e-3)


def test_two_segment_extinction(orc):
    R = radii()
    t1, t2 = 0.7, 2.5
    A1, A2 = t1 * OMEGA * R[1] ** 2, t2 * OMEGA * R[2] ** 2
    L1, L2 = 1e30, 5e30
    F = orc.ray_integrate(NPIX, R, [0, L1, L2, 0], [0, A1, A2, 0])
    g = lambda t: (1 - math.exp(-t)) / t
    ref = g(t1) * L1 / (4 * math.pi * R[1] ** 2) + math.exp(-t1) * g(t2) * L2 / (4 * math.pi * R[2] ** 2)
    assert math.isclose(F, ref, rel_tol=1e-13)
    # segment 0 never extinguishes (tau_thin,0 = 0)
    F0 = orc.ray_integrate(NPIX, R, [0, 0, L2, 0], [1e60, 0, A2, 0])
    assert math.isclose(F0, g(t2) * L2 / (4 * math.pi * R[2] ** 2), rel_tol=1e-13)


def test_compact_thick_body(orc):
    # one thick node (alpha = 1, edge dx, intensity I) at distance r in segment 2:
    # F = omega_thick I = I dx^2 / r^2 (a black body of area dx^2), if it fits the ray
    R = radii()
    I, dx, r = 7.0, 2e15, 1.3 * R[2]
    V = dx ** 3
    beta = R[2] ** 2 / r ** 2
    Lk = [0, 0, I * V, 0]
    Vk = [0, 0, V, 0]
    Qk = [0, 0, beta * V, 0]
    Ak = [0, 0, 50.0 * dx * dx, 0]
    F = orc.ray_integrate(NPIX, R, [0] * 4, [0] * 4, Lk, Ak, Vk, Qk)
    assert math.isclose(F, I * dx * dx / r ** 2, rel_tol=1e-12)
    # behind it, a thin source is dimmed by (1 - f) + f e^(-tau_thick)
    f = (dx * dx / r ** 2) / OMEGA
    tau_k = 50.0 * dx * dx / (dx * dx / r ** 2 * R[2] ** 2)
    Lth = [0, 0, 0, 1e30]
    Ath = [0, 0, 0, 1e-20]
    F2 = orc.ray_integrate(NPIX, R, Lth, Ath, Lk, Ak, Vk, Qk)
    ref = F + ((1 - f) + f * math.exp(-tau_k)) * 1e30 / (4 * math.pi * R[3] ** 2)
    assert math.isclose(F2, ref, rel_tol=1e-12)


def test_merge(orc):
    # flagged pair (1, 2): segment 2 folds into 1 with T = R1^2/R2^2 on L^thin, A^thin
    R = radii()
    L = [0, 2e30, 3e30, 0]
    A = [0, 0.1 * OMEGA * R[1] ** 2, 0.4 * OMEGA * R[2] ** 2, 0]
    F = orc.ray_integrate(NPIX, R, L, A, flag=1 << 1)
    T = R[1] ** 2 / R[2] ** 2
    Lm, Am = L[1] + T * L[2], A[1] + T * A[2]
    tau = Am / (OMEGA * R[1] ** 2)
    ref = (1 - math.exp(-tau)) / tau * Lm / (4 * math.pi * R[1] ** 2)
    assert math.isclose(F, ref, rel_tol=1e-13)
