"""Closed forms and brute-force identities that pin the oracle's walk, mapping,
integration and finalization (Secs. 4.2-4.4)."""
import math
import os

import numpy as np
import pytest

import synth

SIGMA = 5.670374419e-5
HERE = os.path.dirname(os.path.abspath(__file__))


def _leaf_L(t):
    ex = t.export()
    L = np.zeros(t.w.n_leaves)
    m = ex["leaf"] >= 0
    L[ex["leaf"][m]] = ex["vals"][m, 0]
    return L, ex


def test_no_extinction_theta0_equals_brute_force(orc):
    """kappa_ext = 0, theta -> 0: every leaf is accepted; beta R_i^-2 = r^-2 and
    sum_h alpha_h = 1, so J = sum_k L_k / (16 pi^2 r_k^2) (own cell at R_0 = dx/2) and
    F = -sum_k L_k / (4 pi r_k^2) sum_h alpha_kh n^h, for any binning."""
    w = synth.random_uniform(8, seed=3, thick_frac=0.0, kappa_ext_scale=0.0, theta=1e-9)
    t = orc.Tree(w)
    L, _ = _leaf_L(t)
    n, dx = 8, w.box_cm / 8
    cen = synth.cell_centres(n, w.box_cm)
    nhat = np.array([orc.pix2vec(2, h) for h in range(48)])
    targets = np.array([0, 73, 300, 511])
    J, F = t.evaluate(targets)
    for q, tk in enumerate(targets):
        d = cen - cen[tk]
        r2 = (d * d).sum(1)
        r2[tk] = (0.5 * dx) ** 2
        Jb = (L / (16 * math.pi ** 2 * r2)).sum()
        assert math.isclose(J[q], Jb + t.leaves()["jsrc"][tk], rel_tol=1e-12)
        Fb = np.zeros(3)
        for k in range(n ** 3):
            if k == tk:
                continue
            o = np.round(d[k] / dx * 2).astype(np.int64)
            c = orc.alpha_counts(48, orc.alpha_key(o, 2)) / 512.0
            Fb -= L[k] / (4 * math.pi * r2[k]) * (c[:, None] * nhat).sum(0)
        assert np.allclose(F[q], Fb, rtol=1e-11, atol=1e-12 * np.abs(Fb).max())


def test_no_extinction_tree_sum(orc):
    """kappa_ext = 0 at theta = 0.5: J = sum over accepted nodes of L_node / (16 pi^2 r_COL^2)."""
    w = synth.gaussian_clump(16, kappa_ext_scale=0.0)
    t = orc.Tree(w)
    ex = t.export()
    u = t.unit_cm
    for tk in [0, 1234, 2080, 4095]:
        ids = t.accepted(tk)
        own = ex["leaf"][ids] == tk
        c = ex["vals"][ids, 8:11]
        tc = ex["centre"][t.accepted(tk)[own]][0]
        r2 = (((c - tc) * u) ** 2).sum(1)
        r2[own] = (0.5 * w.box_cm / 16) ** 2
        Jb = (ex["vals"][ids, 0] / (16 * math.pi ** 2 * r2)).sum()
        J, _ = t.evaluate([tk])
        assert math.isclose(J[0], Jb, rel_tol=1e-12)


def test_tree_error_within_5_percent(orc):
    """theta = 0.5 against theta -> 0 (every leaf accepted), emission only: within 5 %."""
    w = synth.gaussian_clump(16, kappa_ext_scale=0.0)
    tg = np.arange(0, 4096, 13)
    J, _ = orc.Tree(w).evaluate(tg)
    w.params["theta"] = 1e-9
    J0, _ = orc.Tree(w).evaluate(tg)
    err = np.abs(J / J0 - 1)
    assert err.max() < 0.05


def test_point_source_inverse_square(orc):
    w = synth.point_source(16, kappa0=0.0)
    t = orc.Tree(w)
    J, F = t.evaluate()
    cen = synth.cell_centres(16, w.box_cm)
    host = 8 + 16 * (8 + 16 * 8)
    r2 = ((cen - cen[host]) ** 2).sum(1)
    Lst = w.star_lum[0]
    m = np.arange(16 ** 3) != host
    assert np.allclose(J[m] * 16 * math.pi ** 2 * r2[m] / Lst, 1.0, rtol=1e-12)
    # flux points away from the source, |F| <= L / (4 pi r^2)
    d = cen[m] - cen[host]
    cosang = (F[m] * d).sum(1) / np.linalg.norm(F[m], axis=1) / np.sqrt(r2[m])
    assert cosang.min() > 0.9
    assert (np.linalg.norm(F[m], axis=1) <= Lst / (4 * math.pi * r2[m]) * (1 + 1e-12)).all()


@pytest.mark.parametrize("kappa", [1.0, 10.0])
def test_point_source_extinction_fit(orc, kappa):
    """Fitted kappa from J r^2 along an axis; the paper's own fits are in tests/golden."""
    gold = {}
    for line in open(os.path.join(HERE, "golden", "point_source_extinction.txt")):
        if line.strip() and not line.startswith("#"):
            a, b = line.split()
            gold[float(a)] = float(b)
    n = 32
    w = synth.point_source(n, kappa0=kappa)
    t = orc.Tree(w)
    c = n // 2
    tg = np.array([(c + k) + n * (c + n * c) for k in range(1, n - c)])
    J, _ = t.evaluate(tg)
    r = np.arange(1, n - c) * w.box_cm / n
    slope = np.polyfit(r, np.log(J * r * r), 1)[0]
    kfit = -slope / 1e-18
    # this reading under-extincts by ~9 % at 32^3 (the paper's quadratic bins over-extinct by 3 %)
    assert abs(kfit / kappa - 1) < 0.15
    assert abs(kfit / gold[kappa] - 1) < 0.15


def test_thin_sphere_closed_form(orc):
    """Optically thin uniform sphere: J(centre) = j R, j = (sigma/pi) kappa rho T^4."""
    n = 32
    w = synth.homogeneous(n, 1.0, 1e-22, td=20.0, kappa0=1.0)
    x = synth.cell_centres(n, w.box_cm) - 0.5 * w.box_cm
    R = 0.4 * w.box_cm
    w.rho = np.where((x * x).sum(1) < R * R, 1e-22, 0.0).astype(np.float32)
    c = n // 2
    J, F = orc.Tree(w).evaluate([c + n * (c + n * c)])
    j = SIGMA / math.pi * 1e-22 * 20.0 ** 4
    assert abs(J[0] / (j * R) - 1) < 0.05


def test_long_characteristics_with_extinction(orc):
    """Against brute-force long characteristics through the cells (exact extinction
    along straight lines) on the 16^3 clump with kappa = 1 (central column tau ~ 0.8):
    agreement at the method's accuracy. The method under-extincts (the own segment
    never extinguishes, eq. tauthin), so it lies above the brute force."""
    w = synth.gaussian_clump(16, kappa0=1.0)
    t = orc.Tree(w)
    L, _ = _leaf_L(t)
    lv = t.leaves()
    ak = lv["kappa"] * w.rho.astype(np.float64)
    tg = np.arange(0, 4096, 61)
    J, F = t.evaluate(tg)
    Jb, Fb = orc.brute_lc(16, w.box_cm, L, ak, tg)
    own = L[tg] / (16 * math.pi ** 2 * (0.5 * w.box_cm / 16) ** 2)
    err = J / (Jb + own) - 1
    assert err.min() > 0.0
    assert np.median(err) < 0.06 and err.max() < 0.1


def test_deep_thick_plateau(orc):
    """Inside a large isothermal optically thick region J -> sigma T^4 / pi (App. B)."""
    n = 16
    w = synth.homogeneous(n, 1.0, 1e-17, td=30.0, kappa0=10.0)   # tau per cell ~ 6
    c = n // 2
    J, _ = orc.Tree(w).evaluate([c + n * (c + n * c)])
    assert abs(J[0] / (SIGMA * 30.0 ** 4 / math.pi) - 1) < 0.1


@pytest.mark.parametrize("tau_cell,ncell", [(0.05, 4), (0.2, 8), (0.5, 8), (2.0, 4)])
def test_uniform_slab_closed_form(orc, tau_cell, ncell):
    """An isothermal slab (source function S = sigma T^4 / pi) filling the box laterally,
    empty elsewhere: just outside a face, an infinite slab gives J = (S/2)(1 - E_2(tau))
    and the emergent flux pi S (1 - 2 E_3(tau)). The method mixes extinction within
    segments and the slab is finite (32 cells wide, grazing paths cut off), so the
    measured agreement is stated rather than tight: J 0.82-1.20, |F_z| 0.92-0.96 of the
    infinite-slab values for tau = 0.2-8. Mirror symmetry across the slab is exact."""
    from scipy.special import expn
    n = 32
    w = synth.homogeneous(n, 1.0, 1e-30, td=30.0, kappa0=1.0)
    dx = w.box_cm / n
    z0 = n // 2 - ncell // 2
    rho = np.full((n, n, n), 1e-30, np.float32)
    rho[z0:z0 + ncell] = tau_cell / dx  # kappa = 1
    w.rho = rho.reshape(-1)
    c = n // 2
    below, above = c + n * (c + n * (z0 - 1)), c + n * (c + n * (z0 + ncell))
    J, F = orc.Tree(w).evaluate([below, above])
    tau = tau_cell * ncell
    S = SIGMA * 30.0 ** 4 / math.pi
    Jinf = 0.5 * S * (1.0 - expn(2, tau))
    Finf = math.pi * S * (1.0 - 2.0 * expn(3, tau))
    assert abs(J[0] / J[1] - 1) < 1e-12 and abs(F[0, 2] + F[1, 2]) < 1e-12 * abs(F[1, 2])
    assert F[1, 2] > 0  # radiation leaves the slab upward above it
    assert 0.75 < J[1] / Jinf < 1.25
    assert 0.85 < F[1, 2] / Finf < 1.05


@pytest.mark.parametrize("periodic", [7, 1, 6])
def test_no_extinction_periodic_nearest_copies(orc, periodic):
    """The identity above with periodic axes (Sec. 4.2: only the closest periodic copies
    of a node are considered): every source enters at its nearest copy; a source exactly
    half a box away on a periodic axis has two closest copies, each counted with weight 1/2
    (the reading), so it adds to J but its flux along that axis cancels."""
    n = 8
    w = synth.random_uniform(n, seed=3, thick_frac=0.0, kappa_ext_scale=0.0, theta=1e-9, periodic=periodic)
    t = orc.Tree(w)
    L, _ = _leaf_L(t)
    dx = w.box_cm / n
    cen = synth.cell_centres(n, w.box_cm)
    nhat = np.array([orc.pix2vec(2, h) for h in range(48)])
    targets = np.array([0, 73, 300, 511])
    J, F = t.evaluate(targets)
    for q, tk in enumerate(targets):
        o = np.round((cen - cen[tk]) / dx * 2).astype(np.int64)  # half-cells
        Jb, Fb = t.leaves()["jsrc"][tk], np.zeros(3)
        for k in range(n ** 3):
            if k == tk:
                Jb += L[k] / (16 * math.pi ** 2 * (0.5 * dx) ** 2)
                continue
            copies = [(o[k].copy(), 1.0)]
            for a in range(3):
                if not (periodic >> a) & 1:
                    continue
                nxt = []
                for oc, wt in copies:
                    v = (oc[a] + n) % (2 * n) - n  # into [-n, n) half-cells
                    if v == -n:  # exactly half a box: both copies
                        for s in (-n, n):
                            c2 = oc.copy()
                            c2[a] = s
                            nxt.append((c2, 0.5 * wt))
                    else:
                        oc = oc.copy()
                        oc[a] = v
                        nxt.append((oc, wt))
                copies = nxt
            for oc, wt in copies:
                r2 = ((oc * 0.5 * dx) ** 2).sum()
                Jb += wt * L[k] / (16 * math.pi ** 2 * r2)
                c = orc.alpha_counts(48, orc.alpha_key(oc, 2)) / 512.0
                Fb -= wt * L[k] / (4 * math.pi * r2) * (c[:, None] * nhat).sum(0)
        assert math.isclose(J[q], Jb, rel_tol=1e-12)
        assert np.allclose(F[q], Fb, rtol=1e-11, atol=1e-12 * np.abs(Fb).max())


def test_isotropic_periodic_box_has_no_net_flux(orc):
    """Homogeneous isothermal box, periodic on every axis: with every leaf accepted
    (theta -> 0) each cell sees a point-symmetric set of nearest copies (ties split in
    half), the ray set is antipodally symmetric, so F = 0 to rounding and J is the same in
    every cell. At theta = 0.5 the octree's fixed node boundaries break the symmetry at the
    level of the tree error (measured |F| <= 0.075 x 4 pi J on 16^3); the isolated box
    has cells at its edges that see one side only (|F| up to 0.72 x 4 pi J)."""
    w = synth.homogeneous(8, 1.0, 1e-21, td=20.0, kappa0=5.0, periodic=7, theta=1e-6)
    J, F = orc.Tree(w).evaluate()
    assert np.abs(J / J[0] - 1).max() < 1e-12
    assert (np.linalg.norm(F, axis=1) <= 1e-12 * 4 * math.pi * J).all()
    w = synth.homogeneous(16, 1.0, 1e-21, td=20.0, kappa0=5.0, periodic=7)
    J, F = orc.Tree(w).evaluate()
    assert (np.linalg.norm(F, axis=1) <= 0.1 * 4 * math.pi * J).all()
    w = synth.homogeneous(16, 1.0, 1e-21, td=20.0, kappa0=5.0)
    J, F = orc.Tree(w).evaluate()
    assert (np.linalg.norm(F, axis=1) / (4 * math.pi * J)).max() > 0.5


def test_quadratic_radii_and_ray_matched_theta(orc):
    """Quadratic radii run from R_0 (half the target cell) to R_max with second differences
    constant; the emission-only identity J = sum over accepted nodes of L / (16 pi^2 r^2)
    holds for any radii (beta cancels R_i^2); a negative theta opens nodes down to the
    ray size sqrt(4 pi / N_pix)."""
    w = synth.gaussian_clump(16, kappa_ext_scale=0.0, bin_spacing=1)
    t = orc.Tree(w)
    R = t.radii(0)
    n = len(R) - 1
    assert math.isclose(R[0], 1.0) and math.isclose(R[-1], math.sqrt(3.0) * 32, rel_tol=1e-12)
    d2 = np.diff(R, 2)
    assert np.allclose(d2, d2[0], rtol=1e-9) and d2[0] > 0
    assert np.allclose(R, 1.0 + (R[-1] - 1.0) * (np.arange(n + 1) / n) ** 2, rtol=1e-13)
    Jq, _ = t.evaluate([0, 2080, 4095])
    Jg, _ = orc.Tree(synth.gaussian_clump(16, kappa_ext_scale=0.0)).evaluate([0, 2080, 4095])
    assert np.allclose(Jq, Jg, rtol=1e-12)
    wt = synth.gaussian_clump(16, theta=-1.0)
    w5 = synth.gaussian_clump(16, theta=math.sqrt(4 * math.pi / 48))
    assert np.array_equal(orc.Tree(wt).accepted(2080), orc.Tree(w5).accepted(2080))


def test_col_mapping_identities(orc):
    """Mapping at the centre of luminosity (Sec. 7.6): emission only, J still equals the
    sum over accepted nodes of L / (16 pi^2 r_COL^2) (beta cancels R_i^2 whatever segment
    the COL picks); leaves (COL at the centre) map as before, so with every leaf accepted
    the result equals geometric mapping exactly."""
    w = synth.gaussian_clump(16, kappa_ext_scale=0.0, col_mapping=1)
    t = orc.Tree(w)
    ex = t.export()
    u = t.unit_cm
    for tk in [0, 1234, 2080, 4095]:
        ids = t.accepted(tk)
        own = ex["leaf"][ids] == tk
        c = ex["vals"][ids, 8:11]
        tc = ex["centre"][ids[own]][0]
        r2 = (((c - tc) * u) ** 2).sum(1)
        r2[own] = (0.5 * w.box_cm / 16) ** 2
        J, _ = t.evaluate([tk])
        assert math.isclose(J[0], (ex["vals"][ids, 0] / (16 * math.pi ** 2 * r2)).sum(), rel_tol=1e-12)
    a = orc.Tree(synth.random_uniform(8, seed=2, theta=1e-9, col_mapping=1)).evaluate()
    b = orc.Tree(synth.random_uniform(8, seed=2, theta=1e-9)).evaluate()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_col_mapping_points_flux_at_an_offcentre_source(orc):
    """A lone source off the centre of the nodes that carry it: mapped at the COL, the flux
    seen by distant targets points closer to the true direction than mapped at the
    geometric centres (the reason the paper shifts nodes to their centre of emission)."""
    n = 32
    errs = {}
    for col in (0, 1):
        w = synth.point_source(n, kappa0=0.0, cell=(5, 9, 13), col_mapping=col)
        t = orc.Tree(w)
        cen = synth.cell_centres(n, w.box_cm)
        src = w.star_pos[0]
        tg = np.array([k for k in range(0, n ** 3, 997)])
        _, F = t.evaluate(tg)
        true = cen[tg] - src
        true /= np.linalg.norm(true, axis=1, keepdims=True)
        far = np.linalg.norm(cen[tg] - src, axis=1) > 0.4 * w.box_cm
        cosang = (F[far] * true[far]).sum(1) / np.linalg.norm(F[far], axis=1)
        errs[col] = np.degrees(np.arccos(np.clip(cosang, -1, 1)))
    assert errs[1].mean() < errs[0].mean()
