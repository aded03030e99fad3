"""GB300-native TreeRay/RadPressure hot path.

Thin Python binding of the C ABI in ``include/treeray.h`` (``libtreeray.so``, built
in-tree for sm_103a). Every function marshals arguments only: all steps of the path
run in the library's CUDA kernels. PyTorch provides device memory and streams.
There is no CPU fallback: if the library is missing or no GPU is present the calls
raise.
"""
from __future__ import annotations

import ctypes as C
import os

from .build_lib import OUT as LIB_PATH
from .build_lib import build as build_library

__all__ = ["Params", "Grid", "Context", "Batch", "MLP", "TreeRayError", "lib", "alpha_counts_host",
           "build_library", "LIB_PATH", "STATUS"]

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTBUILT", 5: "ETIMEOUT",
          6: "ENOCONV"}


class TreeRayError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"treeray {STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("npix", C.c_int), ("nbins", C.c_int), ("theta", C.c_double),
                ("kappa_model", C.c_int), ("kappa0", C.c_double), ("dust_to_gas", C.c_double),
                ("dust_emission", C.c_int), ("kappa_ext_scale", C.c_double), ("alpha_s", C.c_int),
                ("periodic", C.c_int), ("bin_spacing", C.c_int), ("col_mapping", C.c_int)]

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        return cls(int(d["npix"]), int(d["nbins"]), float(d["theta"]), int(d["kappa_model"]),
                   float(d["kappa0"]), float(d["dust_to_gas"]), int(d["dust_emission"]),
                   float(d["kappa_ext_scale"]), int(d.get("alpha_s", 8)), int(d.get("periodic", 0)),
                   int(d.get("bin_spacing", 0)), int(d.get("col_mapping", 0)))


class Grid(C.Structure):
    _fields_ = [("n", C.c_int), ("n_blocks", C.c_int), ("blocks", C.POINTER(C.c_int32)),
                ("box", C.c_double)]


_lib = None


def lib():
    """Load libtreeray.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run paper_2204_09072_gb300.build_library()")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32p = C.c_void_p, C.c_int64, C.POINTER(C.c_int32)
    L.treeray_create.argtypes = [C.POINTER(Params), C.POINTER(vp)]
    L.treeray_destroy.argtypes = [vp]
    L.treeray_build.argtypes = [vp, C.POINTER(Grid), vp, vp, vp, C.c_int, vp, vp, vp]
    L.treeray_evaluate.argtypes = [vp, vp, i64, vp, vp, vp]
    L.treeray_radpressure.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.treeray_uv_radpressure.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.treeray_dust_temperature.argtypes = [vp, vp, vp, vp, vp, vp]
    L.treeray_check.argtypes = [vp, vp]
    L.treeray_leaf_count.argtypes = [vp]
    L.treeray_leaf_count.restype = i64
    L.treeray_node_count.argtypes = [vp]
    L.treeray_node_count.restype = i64
    L.treeray_tree_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.treeray_leaf_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.treeray_accepted.argtypes = [vp, vp, i64, C.c_int32, vp, vp, vp]
    L.treeray_alpha_counts_host.argtypes = [C.c_int, C.c_int, vp, i32p]
    L.treeray_alpha_counts_rotated_host.argtypes = [C.c_int, C.c_int, vp, vp, i32p]
    L.treeray_set_orientations.argtypes = [vp, C.c_int, vp, vp]
    L.treeray_walk_stats.argtypes = [vp, vp, i64, vp, vp]
    L.treeray_refresh.argtypes = [vp, vp, vp]
    L.treeray_fixed_point.argtypes = [vp, vp, vp, vp, C.c_int, C.c_double, C.c_int,
                                      C.POINTER(C.c_int), vp]
    L.treeray_autotune.argtypes = [vp, i64, C.POINTER(C.c_int), C.POINTER(C.c_float), vp]
    L.treeray_set_warps_per_target.argtypes = [vp, C.c_int]
    L.treeray_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp)]
    L.treeray_batch_destroy.argtypes = [vp]
    L.treeray_batch_evaluate.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.c_int, vp]
    L.treeray_features.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.treeray_mlp_create.argtypes = [C.c_uint64, C.POINTER(vp)]
    L.treeray_mlp_destroy.argtypes = [vp]
    L.treeray_mlp_set_params.argtypes = [vp, vp, vp]
    L.treeray_mlp_get_params.argtypes = [vp, vp, vp]
    L.treeray_mlp_fit_normalization.argtypes = [vp, vp, vp, i64, vp]
    L.treeray_mlp_train.argtypes = [vp, vp, vp, i64, C.c_int, C.c_int, C.c_float, C.c_uint64, vp, vp]
    L.treeray_mlp_grad.argtypes = [vp, vp, vp, i64, vp, C.POINTER(C.c_float), vp]
    L.treeray_mlp_infer.argtypes = [vp, vp, i64, vp, vp]
    L.treeray_warm_start.argtypes = [vp, vp, vp, vp, vp]
    L.treeray_morton_order_noalloc.argtypes = [C.POINTER(Grid), vp, vp, vp]
    L.treeray_kernel_launches.argtypes = [vp]
    L.treeray_set_walk_stack_limit.argtypes = [vp, C.c_int]
    L.treeray_autotune_launch.argtypes = [vp, i64, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                          C.POINTER(C.c_float), C.POINTER(C.c_float), vp]
    L.treeray_get_launch_config.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.treeray_set_occupancy.argtypes = [vp, C.c_int]
    L.treeray_inject_alloc_failure.argtypes = [vp, C.c_int]
    L.treeray_kernel_launches.restype = i64
    L.treeray_last_error.restype = C.c_char_p
    for f in ("treeray_create", "treeray_destroy", "treeray_build", "treeray_evaluate",
              "treeray_radpressure", "treeray_uv_radpressure", "treeray_dust_temperature", "treeray_check",
              "treeray_tree_export", "treeray_leaf_export", "treeray_accepted",
              "treeray_alpha_counts_host", "treeray_alpha_counts_rotated_host", "treeray_set_orientations",
              "treeray_walk_stats", "treeray_morton_order_noalloc",
              "treeray_refresh", "treeray_fixed_point", "treeray_autotune",
              "treeray_set_warps_per_target", "treeray_batch_create", "treeray_batch_destroy",
              "treeray_batch_evaluate", "treeray_features", "treeray_mlp_create",
              "treeray_mlp_destroy", "treeray_mlp_set_params", "treeray_mlp_get_params",
              "treeray_mlp_fit_normalization", "treeray_mlp_train", "treeray_mlp_grad",
              "treeray_mlp_infer", "treeray_warm_start", "treeray_set_walk_stack_limit",
              "treeray_inject_alloc_failure", "treeray_autotune_launch", "treeray_get_launch_config",
              "treeray_set_occupancy"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _raise(rc: int):
    if rc != 0:
        raise TreeRayError(rc, lib().treeray_last_error().decode())


def _dev(t, dtype, name, allow_none=False):
    """Device pointer of a contiguous CUDA tensor of the given dtype."""
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return C.c_void_p(t.data_ptr())


def _stream(s):
    if s is None:
        import torch
        s = torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def alpha_counts_host(npix: int, s: int, K, rot=None):
    """Angular-kernel hit counts of key K (host-only call, needs no GPU); rot: a 3x3
    rotation of the ray set (C: treeray_alpha_counts_rotated_host)."""
    import numpy as np
    k = np.ascontiguousarray(K, dtype=np.int64)
    out = np.zeros(npix, np.int32)
    if rot is None:
        _raise(lib().treeray_alpha_counts_host(npix, s, C.c_void_p(k.ctypes.data),
                                               out.ctypes.data_as(C.POINTER(C.c_int32))))
    else:
        r = np.ascontiguousarray(rot, dtype=np.float64).reshape(9)
        _raise(lib().treeray_alpha_counts_rotated_host(npix, s, C.c_void_p(k.ctypes.data),
                                                       C.c_void_p(r.ctypes.data),
                                                       out.ctypes.data_as(C.POINTER(C.c_int32))))
    return out


def morton_order_noalloc(box: float, keys, perm, n: int = 0, blocks=None, stream=None):
    """C: treeray_morton_order_noalloc. Morton ordering of the leaves for callers that
    cannot allocate device memory: keys (uint64 viewed as torch.int64) and perm (int32)
    are caller-owned CUDA tensors of the leaf count; the library allocates nothing."""
    import numpy as np
    import torch
    g = Grid()
    g.n = int(n)
    g.box = float(box)
    b = None
    if blocks is not None:
        b = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1)
        g.n_blocks = b.size // 4
        g.blocks = b.ctypes.data_as(C.POINTER(C.c_int32))
    # the kernels write one key and one index per leaf: refuse outputs shorter than that
    n_leaves = int(n) ** 3 if int(n) > 0 else 512 * (0 if b is None else b.size // 4)
    for t, name in ((keys, "keys"), (perm, "perm")):
        if t is not None and t.numel() < n_leaves:
            raise ValueError(f"{name} holds {t.numel()} entries, the grid has {n_leaves} leaves")
    _raise(lib().treeray_morton_order_noalloc(C.byref(g), _dev(keys, torch.int64, "keys"),
                                              _dev(perm, torch.int32, "perm"), _stream(stream)))


class Context:
    """One treeray context (C: treeray_t) on the current CUDA device."""

    def __init__(self, params: dict):
        import torch
        torch.cuda.init()
        self.params = dict(params)
        self._p = Params.from_dict(params)
        h = C.c_void_p()
        _raise(lib().treeray_create(C.byref(self._p), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().treeray_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C: treeray_build
    def build(self, box: float, rho, Td, n: int = 0, blocks=None, kappa=None, star_pos=None,
              star_lum=None, stream=None):
        import numpy as np
        import torch
        g = Grid()
        g.n = int(n)
        g.box = float(box)
        self._blocks = None
        if blocks is not None:
            self._blocks = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1)
            g.n_blocks = self._blocks.size // 4
            g.blocks = self._blocks.ctypes.data_as(C.POINTER(C.c_int32))
        ns = 0 if star_lum is None else len(star_lum)
        sp = np.ascontiguousarray(star_pos if ns else np.zeros((1, 3)), dtype=np.float64).reshape(-1)
        sl = np.ascontiguousarray(star_lum if ns else np.zeros(1), dtype=np.float64)
        _raise(lib().treeray_build(self.h, C.byref(g), _dev(rho, torch.float32, "rho"),
                                   _dev(Td, torch.float32, "Td"),
                                   _dev(kappa, torch.float32, "kappa", True), ns,
                                   C.c_void_p(sp.ctypes.data), C.c_void_p(sl.ctypes.data),
                                   _stream(stream)))

    # -- C: treeray_evaluate
    def evaluate(self, J, F, targets=None, stream=None):
        """C: treeray_evaluate. targets None: every leaf (J has one row per leaf); else one
        row per target (an empty targets tensor is an empty list)."""
        import torch
        n = J.numel() if targets is None else targets.numel()
        if J.numel() < n or F.numel() < 3 * n:
            raise ValueError("J needs n and F 3 n elements")
        _raise(lib().treeray_evaluate(self.h, _dev(targets, torch.int32, "targets", True), n,
                                      _dev(J, torch.float32, "J"), _dev(F, torch.float64, "F"),
                                      _stream(stream)))

    # -- C: treeray_radpressure
    def radpressure(self, J, F, u=None, a_rp=None, force=None, p_src=None, stream=None):
        import torch
        f32 = torch.float32
        _raise(lib().treeray_radpressure(self.h, _dev(J, f32, "J"), _dev(F, torch.float64, "F"),
                                         _dev(u, f32, "u", True), _dev(a_rp, f32, "a_rp", True),
                                         _dev(force, f32, "force", True),
                                         _dev(p_src, f32, "p_src", True), _stream(stream)))

    # -- C: treeray_uv_radpressure
    def uv_radpressure(self, nph, uph, a_uv=None, force_uv=None, x_ion=None, stream=None):
        import torch
        f32 = torch.float32
        _raise(lib().treeray_uv_radpressure(self.h, _dev(nph, f32, "nph"), _dev(uph, f32, "uph"),
                                            _dev(x_ion, f32, "x_ion", True), _dev(a_uv, f32, "a_uv", True),
                                            _dev(force_uv, f32, "force_uv", True), _stream(stream)))

    # -- C: treeray_dust_temperature
    def dust_temperature(self, Tgas, J, Td, heat_extra=None, stream=None):
        import torch
        f32 = torch.float32
        _raise(lib().treeray_dust_temperature(self.h, _dev(Tgas, f32, "Tgas"),
                                              _dev(heat_extra, f32, "heat_extra", True),
                                              _dev(J, f32, "J"), _dev(Td, f32, "Td"),
                                              _stream(stream)))

    # -- C: treeray_refresh
    def refresh(self, Td, stream=None):
        import torch
        _raise(lib().treeray_refresh(self.h, _dev(Td, torch.float32, "Td"), _stream(stream)))

    # -- C: treeray_fixed_point
    def fixed_point(self, Tgas, Td, heat_extra=None, max_iter=200, tol=1e-4, unroll=4,
                    stream=None, raise_on_noconv=True) -> int:
        """Iterate T_d to the fixed point in place; returns the iteration count."""
        import torch
        f32 = torch.float32
        it = C.c_int(0)
        rc = lib().treeray_fixed_point(self.h, _dev(Tgas, f32, "Tgas"),
                                       _dev(heat_extra, f32, "heat_extra", True),
                                       _dev(Td, f32, "Td"), int(max_iter), float(tol), int(unroll),
                                       C.byref(it), _stream(stream))
        if rc == 6 and not raise_on_noconv:
            return -it.value
        _raise(rc)
        return it.value

    # -- C: treeray_autotune
    def autotune(self, n_sample: int = 65536, stream=None):
        """Time 2, 3, 4 and 8 warps per target (3: trees without thick material); keeps the
        fastest. Returns (best, [ms2, ms3, ms4, ms8]), -1 for a choice not tried."""
        best = C.c_int(0)
        ms = (C.c_float * 4)()
        _raise(lib().treeray_autotune(self.h, int(n_sample), C.byref(best), ms, _stream(stream)))
        return best.value, list(ms)

    # -- C: treeray_autotune_launch
    def autotune_launch(self, n_sample: int = 65536, stream=None):
        """Team size, then resident teams per SM; returns (wpt, occupancy_pct, ms over
        2/3/4/8 warps, ms over 100/75/50 % occupancy)."""
        best, occ = C.c_int(0), C.c_int(0)
        ms = (C.c_float * 4)()
        mo = (C.c_float * 3)()
        _raise(lib().treeray_autotune_launch(self.h, int(n_sample), C.byref(best), C.byref(occ), ms, mo,
                                             _stream(stream)))
        return best.value, occ.value, list(ms), list(mo)

    # -- C: treeray_get_launch_config / treeray_set_occupancy
    def launch_config(self):
        w, o = C.c_int(0), C.c_int(0)
        _raise(lib().treeray_get_launch_config(self.h, C.byref(w), C.byref(o)))
        return w.value, o.value

    def set_occupancy(self, pct: int):
        _raise(lib().treeray_set_occupancy(self.h, int(pct)))

    # -- C: treeray_set_orientations
    def set_orientations(self, rot, orient=None):
        """Several HEALPix orientations: rot [k, 3, 3] rotations (host), orient a CUDA
        uint8 tensor of one orientation per leaf (None: leaf mod k). Empty rot: the
        single unturned ray set."""
        import numpy as np
        import torch
        r = np.ascontiguousarray(rot, dtype=np.float64).reshape(-1)
        k = r.size // 9
        self._rot = r
        _raise(lib().treeray_set_orientations(self.h, k, C.c_void_p(r.ctypes.data) if k else None,
                                              _dev(orient, torch.uint8, "orient", allow_none=True)))

    # -- C: treeray_set_warps_per_target
    def set_warps_per_target(self, wpt: int):
        _raise(lib().treeray_set_warps_per_target(self.h, int(wpt)))

    # -- C: treeray_set_walk_stack_limit (test hook)
    def set_walk_stack_limit(self, entries: int):
        _raise(lib().treeray_set_walk_stack_limit(self.h, int(entries)))

    # -- C: treeray_inject_alloc_failure (test hook)
    def inject_alloc_failure(self, n: int):
        _raise(lib().treeray_inject_alloc_failure(self.h, int(n)))

    # -- C: treeray_features
    def features(self, Tgas, phi=None, stream=None):
        """One evaluation with ray optical depths, then the 6 warm-start features per leaf.
        Returns (X [N, 6], J [N], F [3N], tau_mean [N], tau_min [N]) as CUDA tensors."""
        import torch
        n = self.leaf_count
        d = Tgas.device
        X = torch.empty(n * 6, dtype=torch.float32, device=d)
        J = torch.empty(n, dtype=torch.float32, device=d)
        F = torch.empty(3 * n, dtype=torch.float64, device=d)
        tm = torch.empty(n, dtype=torch.float32, device=d)
        tn = torch.empty(n, dtype=torch.float32, device=d)
        f32 = torch.float32
        _raise(lib().treeray_features(self.h, _dev(Tgas, f32, "Tgas"), _dev(phi, f32, "phi", True),
                                      _dev(X, f32, "X"), _dev(J, f32, "J"), _dev(F, torch.float64, "F"),
                                      _dev(tm, f32, "tau_mean"), _dev(tn, f32, "tau_min"), _stream(stream)))
        return X.view(n, 6), J, F, tm, tn

    # -- C: treeray_warm_start
    def warm_start(self, mlp, X, Td, stream=None):
        import torch
        _raise(lib().treeray_warm_start(self.h, mlp.h, _dev(X, torch.float32, "X"),
                                        _dev(Td, torch.float32, "Td"), _stream(stream)))

    # -- C: treeray_check
    def check(self, stream=None):
        _raise(lib().treeray_check(self.h, _stream(stream)))

    @property
    def leaf_count(self) -> int:
        return lib().treeray_leaf_count(self.h)

    @property
    def node_count(self) -> int:
        return lib().treeray_node_count(self.h)

    # -- C: treeray_walk_stats
    def walk_stats(self, targets=None, stream=None):
        """Totals (visited nodes, accepted nodes, angular-kernel entries) over the targets."""
        import torch
        n = self.leaf_count if targets is None else targets.numel()
        tot = torch.zeros(3, dtype=torch.int64, device="cuda")
        _raise(lib().treeray_walk_stats(self.h, _dev(targets, torch.int32, "targets", True), n,
                                        _dev(tot, torch.int64, "totals"), _stream(stream)))
        return tot

    # -- C: treeray_kernel_launches
    @property
    def kernel_launches(self) -> int:
        return lib().treeray_kernel_launches(self.h)

    # -- C: treeray_tree_export
    def tree_export(self, stream=None) -> dict:
        import numpy as np
        nn = self.node_count
        lev = np.zeros(nn, np.int32)
        leaf = np.zeros(nn, np.int32)
        ch = np.zeros(nn, np.int32)
        cen = np.zeros((nn, 3), np.int64)
        vals = np.zeros((nn, 11))
        p = lambda a: C.c_void_p(a.ctypes.data)
        _raise(lib().treeray_tree_export(self.h, p(lev), p(leaf), p(ch), p(cen), p(vals),
                                         _stream(stream)))
        return dict(level=lev, leaf=leaf, child0=ch, centre=cen, vals=vals)

    # -- C: treeray_leaf_export
    def leaf_export(self, stream=None) -> dict:
        import numpy as np
        n = self.leaf_count
        k, t, j, ps = (np.zeros(n) for _ in range(4))
        th = np.zeros(n, np.int32)
        p = lambda a: C.c_void_p(a.ctypes.data)
        _raise(lib().treeray_leaf_export(self.h, p(k), p(t), p(j), p(ps), p(th), _stream(stream)))
        return dict(kappa=k, tau=t, jsrc=j, psrc=ps, thick=th)

    # -- C: treeray_accepted
    def accepted(self, targets, cap: int = 8192, stream=None):
        import torch
        n = targets.numel()
        counts = torch.zeros(n, dtype=torch.int32, device=targets.device)
        ids = torch.full((n, cap), -1, dtype=torch.int32, device=targets.device)
        _raise(lib().treeray_accepted(self.h, _dev(targets, torch.int32, "targets"), n, cap,
                                      _dev(counts, torch.int32, "counts"),
                                      _dev(ids, torch.int32, "ids"), _stream(stream)))
        return counts, ids


class Batch:
    """C: treeray_batch_t. Independent boxes evaluated by one persistent launch."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        h = C.c_void_p()
        _raise(lib().treeray_batch_create(arr, len(self.contexts), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().treeray_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C: treeray_batch_evaluate
    def evaluate(self, Js, Fs, use_graph: bool = True, stream=None):
        import torch
        n = len(self.contexts)
        jp = (C.c_void_p * n)(*[_dev(j, torch.float32, "J").value for j in Js])
        fp = (C.c_void_p * n)(*[_dev(f, torch.float64, "F").value for f in Fs])
        _raise(lib().treeray_batch_evaluate(self.h, jp, fp, int(bool(use_graph)), _stream(stream)))


class MLP:
    """C: treeray_mlp_t. The warm-start network (6 -> 64 -> 64 -> 1, SiLU, BF16/FP32)."""

    N_PARAMS = 4673

    def __init__(self, seed: int = 1):
        h = C.c_void_p()
        _raise(lib().treeray_mlp_create(C.c_uint64(seed), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().treeray_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        import numpy as np
        p = np.zeros(self.N_PARAMS, np.float32)
        nrm = np.zeros(14, np.float32)
        _raise(lib().treeray_mlp_get_params(self.h, C.c_void_p(p.ctypes.data), C.c_void_p(nrm.ctypes.data)))
        return p, nrm

    def set_params(self, params=None, norm=None):
        import numpy as np
        p = None if params is None else np.ascontiguousarray(params, np.float32)
        nrm = None if norm is None else np.ascontiguousarray(norm, np.float32)
        _raise(lib().treeray_mlp_set_params(self.h, None if p is None else C.c_void_p(p.ctypes.data),
                                            None if nrm is None else C.c_void_p(nrm.ctypes.data)))

    def fit_normalization(self, X, y, stream=None):
        import torch
        n = y.numel()
        _raise(lib().treeray_mlp_fit_normalization(self.h, _dev(X, torch.float32, "X"),
                                                   _dev(y, torch.float32, "y"), n, _stream(stream)))

    def train(self, X, y, steps: int, batch: int = 4096, lr: float = 1e-3, seed: int = 1, stream=None):
        import numpy as np
        import torch
        n = y.numel()
        hist = np.zeros(max(steps, 1), np.float32)
        _raise(lib().treeray_mlp_train(self.h, _dev(X, torch.float32, "X"), _dev(y, torch.float32, "y"), n,
                                       int(batch), int(steps), C.c_float(lr), C.c_uint64(seed),
                                       C.c_void_p(hist.ctypes.data), _stream(stream)))
        return hist[:steps]

    def grad(self, X, y, stream=None):
        import numpy as np
        import torch
        g = np.zeros(self.N_PARAMS, np.float32)
        loss = C.c_float(0.0)
        _raise(lib().treeray_mlp_grad(self.h, _dev(X, torch.float32, "X"), _dev(y, torch.float32, "y"),
                                      y.numel(), C.c_void_p(g.ctypes.data), C.byref(loss), _stream(stream)))
        return g, loss.value

    def infer(self, X, stream=None):
        import torch
        n = X.numel() // 6
        y = torch.empty(n, dtype=torch.float32, device=X.device)
        _raise(lib().treeray_mlp_infer(self.h, _dev(X, torch.float32, "X"), n, _dev(y, torch.float32, "y"),
                                       _stream(stream)))
        return y
