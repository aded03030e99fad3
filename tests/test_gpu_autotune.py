"""The autotuner over the evaluate kernel's result-neutral launch choices (team size, then
resident teams per SM) and its process-wide cache keyed by the tree's shape."""
import numpy as np
import pytest

import synth
from gpu_util import build_ctx, evaluate, flux_err

pytestmark = pytest.mark.gpu


def test_autotune_launch_choice_is_cached_and_result_neutral(orc):
    w = synth.random_uniform(32, seed=41, thick_frac=0.0, n_stars=2)
    a, _ = build_ctx(w)
    wpt, occ, ms_w, ms_o = a.autotune_launch(8192)
    assert wpt in (2, 3, 4, 8) and occ in (100, 75, 50)
    assert a.launch_config() == (wpt, occ)
    assert all(m > 0 for m in ms_o) and ms_w[[2, 3, 4, 8].index(wpt)] > 0
    # another context building a tree of the same shape starts from the cached choice
    w2 = synth.random_uniform(32, seed=42, thick_frac=0.0, n_stars=2)
    b, _ = build_ctx(w2)
    assert b.launch_config() == (wpt, occ)
    # a tree of another shape (here: 13 segments, a shape no other test tunes) does not
    c, _ = build_ctx(synth.random_uniform(16, seed=43, thick_frac=0.0, n_stars=2, nbins=13))
    assert c.launch_config() == (4, 100)
    # every occupancy gives the same results (FP32 rounding of the deposits' order) and
    # matches the oracle
    tg = synth.sample_targets(w.n_leaves, 700, seed=44)
    out = []
    for pct in (100, 75, 50, 13):
        a.set_occupancy(pct)
        out.append(evaluate(a, tg))
    for J, F in out[1:]:
        assert np.allclose(J, out[0][0], rtol=1e-6, atol=0)
    Jr, Fr = orc.Tree(w).evaluate(tg)
    assert np.abs(out[-1][0] / Jr - 1).max() <= 1e-4
    assert flux_err(out[-1][1], Fr, Jr).max() <= 1e-4
    for x in (a, b, c):
        x.close()
