"""Host-side checks of the CUDA library that need no GPU: the shared library loads,
exports every entry point declared in include/treeray.h, and its host-built angular
kernel agrees with the oracle's key for key."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def trlib():
    import paper_2204_09072_gb300 as tr
    tr.build_library()
    return tr


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "treeray.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(treeray_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(trlib):
    out = subprocess.run(["nm", "-D", "--defined-only", trlib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (treeray_\w+)", out))
    decl = declared_symbols()
    assert len(decl) >= 14
    missing = [s for s in decl if s not in exported]
    assert not missing, missing
    lib = trlib.lib()
    for s in decl:
        getattr(lib, s)


def test_alpha_table_matches_oracle(trlib, orc):
    rng = np.random.default_rng(0)
    keys = []
    for cls, step, off in [(0, 8, 0), (1, 4, 2), (2, 2, 1), (3, 8, 4)]:
        for _ in range(400):
            keys.append(rng.integers(-5, 6, 3) * step + off if cls else rng.integers(-5, 6, 3) * step)
    for npix in (12, 48, 192):
        for K in keys:
            if not np.any(K):
                continue
            a = trlib.alpha_counts_host(npix, 8, K)
            b = orc.alpha_counts(npix, K, 8)
            assert (a == b).all(), (npix, K)


def test_bad_args_host(trlib):
    with pytest.raises(trlib.TreeRayError):
        trlib.alpha_counts_host(50, 8, [1, 1, 1])


def test_turned_alpha_table_matches_oracle(trlib, orc):
    """Several HEALPix orientations (Sec. 7.6): the library's counts for a turned ray set
    equal the oracle's, key for key, for random rotations and a quarter turn."""
    import synth
    rng = np.random.default_rng(1)
    rots = list(synth.random_rotations(4, seed=31)) + [np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]])]
    keys = []
    for step, off in [(8, 0), (4, 2), (2, 1), (8, 4)]:
        for _ in range(60):
            keys.append(rng.integers(-6, 7, 3) * step + off)
    for npix in (12, 48, 192):
        for R in rots:
            for K in keys:
                if not np.any(K):
                    continue
                a = trlib.alpha_counts_host(npix, 8, K, rot=R)
                b = orc.alpha_counts(npix, K, 8, rot=R)
                assert (a == b).all(), (npix, K)
                assert a.sum() == 512


def test_noalloc_rejects_negative_n_before_any_launch(trlib):
    """A negative n is neither a uniform grid nor an AMR grid: the call returns EINVAL
    during argument checking, before any CUDA call (so this runs without a GPU)."""
    import ctypes as C
    g = trlib.Grid()
    g.n = -1
    g.n_blocks = 1
    blocks = (C.c_int32 * 4)(0, 0, 0, 3)
    g.blocks = C.cast(blocks, C.POINTER(C.c_int32))
    g.box = 1.0
    # never dereferenced: the grid is rejected first
    rc = trlib.lib().treeray_morton_order_noalloc(C.byref(g), C.c_void_p(256), C.c_void_p(512), None)
    assert rc == 1
    assert b"n must be" in trlib.lib().treeray_last_error()


def test_noalloc_wrapper_checks_output_length(trlib):
    """The binding refuses key/permutation outputs shorter than the leaf count (the kernels
    write one entry per leaf), for uniform and AMR grids, before calling the library."""
    import torch
    short = torch.empty(7, dtype=torch.int64)
    ok = torch.empty(8, dtype=torch.int32)
    with pytest.raises(ValueError, match="keys holds 7"):
        trlib.morton_order_noalloc(1.0, short, ok, n=2)
    blocks = np.array([[0, 0, 0, 3], [0, 0, 0, 3]], np.int32)
    with pytest.raises(ValueError, match="perm holds 8"):
        trlib.morton_order_noalloc(1.0, torch.empty(1024, dtype=torch.int64), ok, blocks=blocks)
