"""Python driver of the FP64 CPU oracle (``oracle/treeray_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference legs of bench.py may import this package; the CUDA
product path never does. The C source is compiled with gcc (``-O2 -fopenmp
-ffp-contract=off``) into ``oracle/liboracle.so`` on first use.

What each function computes, and which part of the paper it follows, is stated
in the C source beside the function.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "treeray_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (skipped when up to date)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("npix", C.c_int), ("nbins", C.c_int), ("theta", C.c_double),
                ("kappa_model", C.c_int), ("kappa0", C.c_double), ("dust_to_gas", C.c_double),
                ("dust_emission", C.c_int), ("kappa_ext_scale", C.c_double), ("alpha_s", C.c_int),
                ("periodic", C.c_int), ("bin_spacing", C.c_int), ("col_mapping", C.c_int)]


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.POINTER
            L.or_build.argtypes = [P(_Params), C.c_int, C.c_double, C.c_int64, P(C.c_int32),
                                   P(C.c_int32), P(C.c_float), P(C.c_float), P(C.c_float), C.c_int,
                                   P(C.c_double), P(C.c_double), P(C.c_void_p)]
            L.or_build.restype = C.c_int
            L.or_tree_free.argtypes = [C.c_void_p]
            L.or_evaluate.argtypes = [C.c_void_p, C.c_int64, P(C.c_int64), P(C.c_double),
                                      P(C.c_double), C.c_int]
            L.or_evaluate.restype = C.c_int
            L.or_radpressure.argtypes = [C.c_void_p, C.c_int64, P(C.c_int64), P(C.c_double),
                                         P(C.c_double), P(C.c_double), P(C.c_double),
                                         P(C.c_double), P(C.c_double)]
            L.or_uv_radpressure.argtypes = [C.c_void_p, C.c_int64, P(C.c_int64), P(C.c_double),
                                            P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double)]
            L.or_dust_temperature.argtypes = [P(_Params), C.c_int64, P(C.c_float), P(C.c_float),
                                              P(C.c_float), P(C.c_double), P(C.c_float),
                                              P(C.c_double)]
            L.or_td_solve.argtypes = [P(_Params), C.c_double, C.c_double, C.c_double, C.c_double,
                                      P(C.c_float), C.c_int64]
            L.or_td_solve.restype = C.c_double
            L.or_tree_nnodes.argtypes = [C.c_void_p]
            L.or_tree_nnodes.restype = C.c_int64
            L.or_tree_export.argtypes = [C.c_void_p, P(C.c_int32), P(C.c_int32), P(C.c_int32),
                                         P(C.c_int64), P(C.c_double)]
            L.or_leaf_export.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double), P(C.c_double),
                                         P(C.c_double), P(C.c_int32)]
            L.or_accepted.argtypes = [C.c_void_p, C.c_int64, P(C.c_int32), C.c_int64]
            L.or_accepted.restype = C.c_int64
            L.or_walk_stats.argtypes = [C.c_void_p, C.c_int64, P(C.c_int64)]
            L.or_target_radii.argtypes = [C.c_void_p, C.c_int64, P(C.c_double)]
            L.or_alpha_key.argtypes = [P(C.c_int64), C.c_int64, P(C.c_int64)]
            L.or_alpha_counts.argtypes = [C.c_int, C.c_int, P(C.c_int64), P(C.c_int)]
            L.or_alpha_counts_rot.argtypes = [C.c_int, C.c_int, P(C.c_int64), P(C.c_double),
                                              P(C.c_int)]
            L.or_set_orientations.argtypes = [C.c_void_p, C.c_int, P(C.c_double), P(C.c_uint8)]
            L.or_set_orientations.restype = C.c_int
            L.or_ang2pix.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
            L.or_ang2pix.restype = C.c_int
            L.or_pix2vec.argtypes = [C.c_int, C.c_int, P(C.c_double)]
            L.or_unit_cm.argtypes = [C.c_void_p]
            L.or_unit_cm.restype = C.c_double
            L.or_ray_integrate.argtypes = [C.c_int, C.c_int] + [P(C.c_double)] * 7 + [C.c_uint64]
            L.or_ray_integrate.restype = C.c_double
            L.or_brute_lc.argtypes = [C.c_int, C.c_double, P(C.c_double), P(C.c_double), C.c_int64,
                                      P(C.c_int64), C.c_int, P(C.c_double), P(C.c_double)]
            _lib = L
    return _lib


def make_params(d: dict) -> _Params:
    return _Params(int(d["npix"]), int(d["nbins"]), float(d["theta"]), int(d["kappa_model"]),
                   float(d["kappa0"]), float(d["dust_to_gas"]), int(d["dust_emission"]),
                   float(d["kappa_ext_scale"]), int(d.get("alpha_s", 8)), int(d.get("periodic", 0)),
                   int(d.get("bin_spacing", 0)), int(d.get("col_mapping", 0)))


# ---------------------------------------------------------------- HEALPix / alpha

def ang2pix(nside: int, v) -> int:
    return lib().or_ang2pix(nside, float(v[0]), float(v[1]), float(v[2]))


def pix2vec(nside: int, pix: int) -> np.ndarray:
    out = np.zeros(3)
    lib().or_pix2vec(nside, pix, _p(out, C.c_double))
    return out


def alpha_key(o, E: int) -> np.ndarray:
    o = np.ascontiguousarray(o, dtype=np.int64)
    K = np.zeros(3, np.int64)
    lib().or_alpha_key(_p(o, C.c_int64), int(E), _p(K, C.c_int64))
    return K


def alpha_counts(npix: int, K, s: int = 8, rot=None) -> np.ndarray:
    """Angular-kernel hit counts of key K; rot: a 3x3 rotation of the ray set."""
    K = np.ascontiguousarray(K, dtype=np.int64)
    out = np.zeros(npix, np.int32)
    if rot is None:
        lib().or_alpha_counts(npix, s, _p(K, C.c_int64), _p(out, C.c_int))
    else:
        R = np.ascontiguousarray(rot, dtype=np.float64).reshape(9)
        lib().or_alpha_counts_rot(npix, s, _p(K, C.c_int64), _p(R, C.c_double), _p(out, C.c_int))
    return out


def ray_integrate(npix: int, R_cm, Lth, Ath, Lk=None, Ak=None, Vk=None, Qk=None, flag: int = 0):
    nb = len(Lth)
    z = np.zeros(nb)
    arr = [np.array(a if a is not None else z, dtype=np.float64) for a in (Lth, Ath, Lk, Ak, Vk, Qk)]
    R = np.ascontiguousarray(R_cm, dtype=np.float64)
    return lib().or_ray_integrate(nb, npix, *[_p(a, C.c_double) for a in arr], _p(R, C.c_double),
                                  C.c_uint64(flag))


# ---------------------------------------------------------------------- tree

class Tree:
    """Oracle tree for one workload (see ``synth.Workload``)."""

    def __init__(self, w, params: dict | None = None):
        self.w = w
        self.params = dict(w.params if params is None else params)
        self._p = make_params(self.params)
        L = lib()
        handle = C.c_void_p()
        self._keep = [np.ascontiguousarray(w.leaf_level, np.int32),
                      np.ascontiguousarray(w.leaf_ijk, np.int32).reshape(-1),
                      np.ascontiguousarray(w.rho, np.float32),
                      np.ascontiguousarray(w.td, np.float32),
                      None if w.kappa is None else np.ascontiguousarray(w.kappa, np.float32),
                      np.ascontiguousarray(w.star_pos, np.float64).reshape(-1),
                      np.ascontiguousarray(w.star_lum, np.float64)]
        lev, ijk, rho, td, kap, sp, sl = self._keep
        rc = L.or_build(C.byref(self._p), int(w.lmax), float(w.box_cm), int(w.n_leaves),
                        _p(lev, C.c_int32), _p(ijk, C.c_int32), _p(rho, C.c_float),
                        _p(td, C.c_float), _p(kap, C.c_float), int(len(sl)), _p(sp, C.c_double),
                        _p(sl, C.c_double), C.byref(handle))
        if rc != 0:
            raise ValueError(f"oracle build failed ({rc})")
        self.h = handle

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().or_tree_free(self.h)
                self.h = None
        except Exception:
            pass

    @property
    def n_nodes(self) -> int:
        return lib().or_tree_nnodes(self.h)

    @property
    def unit_cm(self) -> float:
        return lib().or_unit_cm(self.h)

    def evaluate(self, targets=None, threads: int = 0):
        n = self.w.n_leaves
        t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
        J = np.zeros(len(t))
        F = np.zeros((len(t), 3))
        rc = lib().or_evaluate(self.h, len(t), _p(t, C.c_int64), _p(J, C.c_double),
                               _p(F, C.c_double), int(threads))
        if rc != 0:
            raise RuntimeError(f"oracle evaluate failed ({rc})")
        return J, F

    def set_orientations(self, rot, orient=None):
        """Several HEALPix orientations: rot [k, 3, 3] rotations, orient [n_leaves] uint8
        (None: leaf mod k). An empty rot goes back to the single unturned ray set."""
        R = np.ascontiguousarray(rot, dtype=np.float64).reshape(-1)
        k = len(R) // 9
        o = None if orient is None else np.ascontiguousarray(orient, np.uint8)
        self._orient = (R, o)
        rc = lib().or_set_orientations(self.h, k, _p(R, C.c_double) if k else None, _p(o, C.c_uint8))
        if rc != 0:
            raise ValueError("bad orientations")

    def radpressure(self, J, F, targets=None):
        n = len(J)
        t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
        J = np.ascontiguousarray(J, np.float64)
        F = np.ascontiguousarray(F, np.float64).reshape(-1)
        u = np.zeros(n)
        a = np.zeros(3 * n)
        f = np.zeros(3 * n)
        ps = np.zeros(n)
        lib().or_radpressure(self.h, n, _p(t, C.c_int64), _p(J, C.c_double), _p(F, C.c_double),
                             _p(u, C.c_double), _p(a, C.c_double), _p(f, C.c_double),
                             _p(ps, C.c_double))
        return u, a.reshape(n, 3), f.reshape(n, 3), ps

    def uv_radpressure(self, nph, uph, x_ion=None, targets=None):
        """UV radiation pressure (App. C) per leaf: returns a_uv [n, 3], force [n, 3]."""
        n = len(nph)
        t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
        nph = np.ascontiguousarray(nph, np.float64)
        uph = np.ascontiguousarray(uph, np.float64).reshape(-1)
        x = None if x_ion is None else np.ascontiguousarray(x_ion, np.float64)
        a = np.zeros(3 * n)
        f = np.zeros(3 * n)
        lib().or_uv_radpressure(self.h, n, _p(t, C.c_int64), _p(nph, C.c_double), _p(uph, C.c_double),
                                _p(x, C.c_double), _p(a, C.c_double), _p(f, C.c_double))
        return a.reshape(n, 3), f.reshape(n, 3)

    def export(self):
        nn = self.n_nodes
        lev = np.zeros(nn, np.int32)
        leaf = np.zeros(nn, np.int32)
        ch = np.zeros(nn, np.int32)
        cen = np.zeros((nn, 3), np.int64)
        vals = np.zeros((nn, 11))
        lib().or_tree_export(self.h, _p(lev, C.c_int32), _p(leaf, C.c_int32), _p(ch, C.c_int32),
                             _p(cen, C.c_int64), _p(vals, C.c_double))
        return dict(level=lev, leaf=leaf, child0=ch, centre=cen, vals=vals)

    def leaves(self):
        n = self.w.n_leaves
        k, t, j, p = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
        th = np.zeros(n, np.int32)
        lib().or_leaf_export(self.h, _p(k, C.c_double), _p(t, C.c_double), _p(j, C.c_double),
                             _p(p, C.c_double), _p(th, C.c_int32))
        return dict(kappa=k, tau=t, jsrc=j, psrc=p, thick=th)

    def accepted(self, leaf: int) -> np.ndarray:
        cap = 1 << 20
        ids = np.zeros(cap, np.int32)
        n = lib().or_accepted(self.h, int(leaf), _p(ids, C.c_int32), cap)
        return ids[:min(n, cap)].copy()

    def walk_stats(self, leaf: int) -> np.ndarray:
        """(visited nodes, accepted nodes, angular-kernel entries) of one target's walk."""
        out = np.zeros(3, np.int64)
        lib().or_walk_stats(self.h, int(leaf), _p(out, C.c_int64))
        return out

    def radii(self, leaf: int) -> np.ndarray:
        R = np.zeros(self.params["nbins"] + 1)
        lib().or_target_radii(self.h, int(leaf), _p(R, C.c_double))
        return R


def dust_temperature(params: dict, rho, tgas, J, heat=None, kappa=None) -> np.ndarray:
    p = make_params(params)
    n = len(rho)
    rho = np.ascontiguousarray(rho, np.float32)
    tgas = np.ascontiguousarray(tgas, np.float32)
    J = np.ascontiguousarray(J, np.float64)
    heat = None if heat is None else np.ascontiguousarray(heat, np.float32)
    kappa = None if kappa is None else np.ascontiguousarray(kappa, np.float32)
    out = np.zeros(n)
    lib().or_dust_temperature(C.byref(p), n, _p(rho, C.c_float), _p(tgas, C.c_float),
                              _p(heat, C.c_float), _p(J, C.c_double), _p(kappa, C.c_float),
                              _p(out, C.c_double))
    return out


def td_solve(params: dict, rho: float, tgas: float, J: float, heat: float = 0.0) -> float:
    p = make_params(params)
    return lib().or_td_solve(C.byref(p), rho, tgas, J, heat, None, 0)


def brute_lc(n: int, box: float, Lcell, ak, targets, with_ext: bool = True):
    Lcell = np.ascontiguousarray(Lcell, np.float64)
    ak = np.ascontiguousarray(ak, np.float64)
    t = np.ascontiguousarray(targets, np.int64)
    J = np.zeros(len(t))
    F = np.zeros((len(t), 3))
    lib().or_brute_lc(n, box, _p(Lcell, C.c_double), _p(ak, C.c_double), len(t), _p(t, C.c_int64),
                      int(with_ext), _p(J, C.c_double), _p(F, C.c_double))
    return J, F


def fixed_point(w, tgas, td0, heat=None, max_iter: int = 200, tol: float = 1e-4, threads: int = 0):
    """Dust-temperature / IR-field fixed point (Sec. 4.6 balance iterated with the
    transfer solution): T_d -> tree -> J -> T_new until max |T_new - T_d| / T_d < tol.
    T_d is kept in float32 between iterations, as the inputs of the method are FP32
    fields. Returns (T_d float32, iterations, list of per-iteration max changes)."""
    import copy
    ww = copy.copy(w)
    td = np.ascontiguousarray(td0, np.float32).copy()
    hist = []
    for it in range(1, max_iter + 1):
        ww.td = td
        J, _ = Tree(ww).evaluate(threads=threads)
        tn = dust_temperature(ww.params, ww.rho, tgas, J.astype(np.float32).astype(np.float64), heat,
                              ww.kappa).astype(np.float32)
        rel = float(np.max(np.abs(tn.astype(np.float64) - td) / td))
        hist.append(rel)
        td = tn
        if rel < tol:
            return td, it, hist
    return td, -max_iter, hist
