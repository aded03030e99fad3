"""The optically thick blob suite (S, M, L, S-, S+ on 64^3 cells) on the GPU against the
FP64 oracle: leaf quantities and the tree (S- has cells without any material), and J/F on
a ragged sample of targets plus every cell inside the blob."""
import numpy as np
import pytest

import synth
from gpu_util import build_ctx, evaluate, flux_err

pytestmark = pytest.mark.gpu

PC = 3.0857e18


@pytest.mark.parametrize("variant", ["S", "M", "L", "S-", "S+"])
def test_blob_suite(orc, variant):
    w = synth.blob_suite(variant, 64)
    t = orc.Tree(w)
    ctx, _ = build_ctx(w)
    o, g = t.leaves(), ctx.leaf_export()
    for k in ("kappa", "tau", "thick"):
        assert (g[k] == o[k]).all(), k
    oe, ge = t.export(), ctx.tree_export()
    for k in ("level", "leaf", "child0", "centre"):
        assert (ge[k] == oe[k]).all(), k
    assert np.allclose(ge["vals"], oe["vals"], rtol=1e-14, atol=0)
    cen = synth.cell_centres(64, w.box_cm) - 0.5 * w.box_cm
    r = np.sqrt((cen ** 2).sum(1))
    R = 0.5 * synth.BLOB_DIAMETER_PC[variant[0]] * PC
    tg = np.union1d(synth.sample_targets(w.n_leaves, 2001, seed=12), np.nonzero(r < R + 0.5 * PC)[0])
    J, F = evaluate(ctx, tg)
    Jr, Fr = t.evaluate(tg)
    assert np.abs(J / Jr - 1).max() <= 1e-4
    assert flux_err(F, Fr, Jr).max() <= 1e-4
