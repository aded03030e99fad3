"""The no-allocation Morton-ordering entry point (treeray_morton_order_noalloc).

It serves callers that cannot call cudaMalloc, for example a host code whose own pool
allocator owns all device memory: all its scratch lives in one fixed array inside the
library. The test calls it through the C ABI twice in a row on each of two grids, in
an order that leaves the shared scratch holding the other grid's data, and checks the
leaf order against the one the regular tree build produces (bit-exact, as for all
integer work). The file is collected last so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _build_order(w):
    """Leaf order of the regular build: leaf ids of the tree's leaves, level by level."""
    from gpu_util import build_ctx
    ctx, _ = build_ctx(w)
    ex = ctx.tree_export()
    leaf = ex["leaf"] >= 0
    order = []
    for lv in np.unique(ex["level"][leaf]):
        m = leaf & (ex["level"] == lv)
        order.append(ex["leaf"][m])
    ctx.close()
    return np.concatenate(order)


def _noalloc(w):
    import torch

    import paper_2204_09072_gb300 as tr
    n = w.n_leaves
    keys = torch.full((n,), -1, dtype=torch.int64, device="cuda:0")
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    tr.morton_order_noalloc(w.box_cm, keys, perm, n=w.uniform_n, blocks=w.blocks)
    torch.cuda.synchronize()
    return keys.cpu().numpy(), perm.cpu().numpy()


def test_noalloc_order_matches_build_twice():
    import paper_2204_09072_gb300 as tr
    tr.build_library()
    grids = [synth.random_uniform(32, seed=4),
             synth.amr_core(n_base_blocks=2, max_level=2, target_leaves=40 * 512, n_stars=1)]
    refs = [_build_order(w) for w in grids]
    for rep in range(2):
        for w, ref in zip(grids, refs):
            keys, perm = _noalloc(w)
            assert (perm == ref).all(), (w.name, rep)
            k = keys.view(np.uint64)
            assert (np.diff(k.astype(np.float64)) >= 0).all() and (k[1:] != k[:-1]).all()


def test_noalloc_rejects_too_many_leaves():
    """Through the C ABI directly (the binding would refuse the short outputs first): a grid
    beyond the fixed scratch size returns EINVAL before anything is written."""
    import ctypes as C

    import torch

    import paper_2204_09072_gb300 as tr
    keys = torch.empty(1, dtype=torch.int64, device="cuda:0")
    perm = torch.empty(1, dtype=torch.int32, device="cuda:0")
    g = tr.Grid()
    g.n = 128   # 2097152 leaves > 524288
    g.box = 1.0
    rc = tr.lib().treeray_morton_order_noalloc(C.byref(g), C.c_void_p(keys.data_ptr()),
                                               C.c_void_p(perm.data_ptr()), None)
    assert rc == 1 and b"524288" in tr.lib().treeray_last_error()
    with pytest.raises(ValueError, match="2097152 leaves"):
        tr.morton_order_noalloc(1.0, keys, perm, n=128)


def test_noalloc_uniform_grid_under_capture_and_amr_refused():
    """A uniform grid needs no host copy, so its ordering can be recorded into a CUDA graph
    and replayed; an AMR grid copies its block table from the host on each call, which a
    capture cannot hold, and is refused with EINVAL while the stream is capturing."""
    import torch

    import paper_2204_09072_gb300 as tr
    w = synth.random_uniform(16, seed=6)
    ref = _build_order(w)
    _noalloc(w)  # the first call on the device (address look-up) precedes the capture
    n = w.n_leaves
    keys = torch.full((n,), -1, dtype=torch.int64, device="cuda:0")
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        tr.morton_order_noalloc(w.box_cm, keys, perm, n=w.uniform_n, stream=s)
    perm.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    assert (perm.cpu().numpy() == ref).all()

    a = synth.amr_core(n_base_blocks=2, max_level=2, target_leaves=40 * 512, n_stars=1)
    ka = torch.empty(a.n_leaves, dtype=torch.int64, device="cuda:0")
    pa = torch.empty(a.n_leaves, dtype=torch.int32, device="cuda:0")
    g2 = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.stream(s):
        g2.capture_begin()
        try:
            tr.morton_order_noalloc(a.box_cm, ka, pa, blocks=a.blocks, stream=s)
        except tr.TreeRayError as e:
            err = e
        finally:
            g2.capture_end()
    assert err is not None and err.code == 1 and "captured" in str(err)
