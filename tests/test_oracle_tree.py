"""Tree structure and node-moment pins for the oracle (Sec. 4.1, App. A)."""
import numpy as np

import synth


def test_uniform_tree_shape_and_sums(orc):
    w = synth.random_uniform(8, seed=1)
    t = orc.Tree(w)
    ex = t.export()
    L = 3
    assert t.n_nodes == sum(8 ** l for l in range(L + 1))
    for l in range(L + 1):
        assert (ex["level"] == l).sum() == 8 ** l
    leaves = ex["leaf"] >= 0
    assert leaves.sum() == 512 and (ex["level"][leaves] == L).all()
    v = ex["vals"]
    # every h-node's sums equal the sums over its 8 sub-nodes
    for i in np.where(~leaves)[0]:
        c0 = ex["child0"][i]
        for q in range(7):
            assert np.isclose(v[i, q], v[c0:c0 + 8, q].sum(), rtol=1e-13, atol=0)
    # root sums equal direct sums over leaves: mass and volumes
    dx = w.box_cm / 8
    assert np.isclose(v[0, 6], (w.rho.astype(np.float64) * dx ** 3).sum(), rtol=1e-12)
    assert np.isclose(v[0, 2] + v[0, 5], w.box_cm ** 3, rtol=1e-12)
    lv = t.leaves()
    thick = lv["thick"].astype(bool)
    assert np.isclose(v[0, 5], thick.sum() * dx ** 3, rtol=1e-12)
    assert thick.any() and (~thick).any()


def test_thin_luminosity_closed_form(orc):
    # thin b-node: L = 4 sigma rho kappa T^4 dV equals 4 pi x emission coefficient x volume
    w = synth.homogeneous(4, 1.0, 1e-22, td=25.0, kappa0=3.0)
    t = orc.Tree(w)
    v = t.export()["vals"]
    dx = w.box_cm / 4
    sigma = 5.670374419e-5
    j = sigma / np.pi * 3.0 * float(np.float32(1e-22)) * 25.0 ** 4  # j = (sigma/pi) kappa rho T^4
    assert np.isclose(v[0, 0], 4 * np.pi * j * w.box_cm ** 3, rtol=1e-12)


def test_col_symmetric_and_point(orc):
    w = synth.gaussian_clump(8)
    t = orc.Tree(w)
    ex = t.export()
    # symmetric clump: root COL at the box centre (8 half-units)
    assert np.allclose(ex["vals"][0, 8:11], ex["centre"][0], atol=1e-9)
    # point source alone: every ancestor's COL sits at the host cell centre
    w = synth.point_source(8, cell=(5, 2, 6))
    t = orc.Tree(w)
    ex = t.export()
    host = np.array([11, 5, 13])
    anc = 0
    for i in range(t.n_nodes):
        if ex["leaf"][i] < 0 and ex["vals"][i, 0] > 0:
            anc += 1
            assert np.allclose(ex["vals"][i, 8:11], host, rtol=0, atol=1e-12)
        elif ex["leaf"][i] < 0:
            # no luminosity: COL falls back to the geometric centre
            assert np.allclose(ex["vals"][i, 8:11], ex["centre"][i], rtol=0, atol=0)
    assert anc == 3


def test_amr_tree(orc):
    w = synth.amr_core(n_base_blocks=2, max_level=1, target_leaves=8 * 512, n_stars=2)
    t = orc.Tree(w)
    ex = t.export()
    assert (ex["leaf"] >= 0).sum() == w.n_leaves
    # every h-node has exactly 8 sub-nodes and sums match
    v = ex["vals"]
    for i in np.where(ex["leaf"] < 0)[0]:
        c0 = ex["child0"][i]
        assert (ex["level"][c0:c0 + 8] == ex["level"][i] + 1).all()
        assert np.isclose(v[i, 6], v[c0:c0 + 8, 6].sum(), rtol=1e-13)
    dx = w.box_cm / 2.0 ** w.leaf_level
    assert np.isclose(v[0, 6], (w.rho.astype(np.float64) * dx ** 3).sum(), rtol=1e-12)
