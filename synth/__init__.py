"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module only makes input fields (grid structure, density, dust temperature,
star particles) with numpy's PCG64 generator. It holds none of the transfer
method's arithmetic: opacities, luminosities, trees, rays and all derived
quantities are computed separately by the oracle and by the CUDA library.

Shapes follow the paper's test problems and its collapsing-core run:
a Gaussian clump on a uniform grid, a lognormal turbulent cloud with a central
star, homogeneous media with a point source (the point-source benchmark of the
paper's benchmark section), an optically thick blob, and an AMR octree of 8^3-cell
blocks around a collapsing core.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PC_CM = 3.0857e18
LSUN = 3.828e33
MSUN = 1.989e33


@dataclasses.dataclass
class Workload:
    """A grid of leaf cells plus the fields the method needs.

    Leaves are listed in the caller's order: x-fastest for uniform grids,
    block-major then x-fastest inside each 8^3 block for AMR grids.
    ``leaf_level[k]`` is the octree level of leaf k (root = level 0, edge
    box / 2**level) and ``leaf_ijk[k]`` its integer coordinates at that level.
    """
    name: str
    box_cm: float
    lmax: int
    leaf_level: np.ndarray          # int32[N]
    leaf_ijk: np.ndarray            # int32[N, 3]
    rho: np.ndarray                 # float32[N], g/cm^3
    td: np.ndarray                  # float32[N], K
    kappa: np.ndarray | None = None  # float32[N], cm^2/g (None: use the params' model)
    star_pos: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 3)))
    star_lum: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0,)))
    tgas: np.ndarray | None = None   # float32[N], K
    phi: np.ndarray | None = None    # float32[N], ionising photon flux (photons/s/cm^2)
    heat_extra: np.ndarray | None = None  # float32[N], erg/s/cm^3
    params: dict = dataclasses.field(default_factory=dict)
    uniform_n: int = 0               # n for an n^3 uniform grid, 0 for AMR
    blocks: np.ndarray | None = None  # int32[nb, 4] (bi, bj, bk, cell level) for AMR

    @property
    def n_leaves(self) -> int:
        return int(self.rho.shape[0])


def default_params(**over) -> dict:
    p = dict(npix=48, nbins=20, theta=0.5, kappa_model=0, kappa0=5.0,
             dust_to_gas=0.01, dust_emission=1, kappa_ext_scale=1.0, alpha_s=8, periodic=0)
    p.update(over)
    return p


def uniform_structure(n: int):
    """Leaf levels and coordinates of an n^3 uniform grid, x fastest."""
    lmax = int(round(math.log2(n)))
    if 1 << lmax != n:
        raise ValueError("n must be a power of two")
    k = np.arange(n ** 3, dtype=np.int64)
    ijk = np.stack([k % n, (k // n) % n, k // (n * n)], axis=1).astype(np.int32)
    lev = np.full(n ** 3, lmax, dtype=np.int32)
    return lmax, lev, ijk


def cell_centres(n: int, box_cm: float) -> np.ndarray:
    lmax, _, ijk = uniform_structure(n)
    return (ijk.astype(np.float64) + 0.5) * (box_cm / n)


def _grf(n: int, slope: float, rng: np.random.Generator) -> np.ndarray:
    """Gaussian random field with P(k) ~ k^slope on an n^3 periodic grid, unit variance.

    Indexed [z, y, x] and returned flattened x-fastest.
    """
    white = rng.standard_normal((n, n, n))
    fk = np.fft.rfftn(white)
    kz = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kx = np.fft.rfftfreq(n)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)   # sqrt(P) = k^(slope/2)
    amp[0, 0, 0] = 0.0
    g = np.fft.irfftn(fk * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g.reshape(-1)


def gaussian_clump(n: int = 32, box_pc: float = 1.0, kappa0: float = 5.0,
                   td: float = 20.0, **pover) -> Workload:
    """Gaussian clump rho0 (1 + 99 exp(-r^2 / (2 (0.1 pc)^2))) on rho0 = 1e-20 g/cm^3."""
    box = box_pc * PC_CM
    lmax, lev, ijk = uniform_structure(n)
    x = cell_centres(n, box) - 0.5 * box
    r2 = (x * x).sum(1)
    s = 0.1 * PC_CM
    rho = 1e-20 * (1.0 + 99.0 * np.exp(-r2 / (2 * s * s)))
    return Workload(name=f"clump{n}", box_cm=box, lmax=lmax, leaf_level=lev, leaf_ijk=ijk,
                    rho=rho.astype(np.float32), td=np.full(n ** 3, td, np.float32),
                    params=default_params(kappa_model=0, kappa0=kappa0, **pover), uniform_n=n)


def turbulent_cloud(n: int = 128, box_pc: float = 2.0, sigma_ln: float = 1.5,
                    mean_rho: float = 1e-20, seed: int = 2, t_seed: int = 3,
                    n_stars: int = 1, star_lum_lsun: float = 1e5, **pover) -> Workload:
    """Lognormal turbulent density (P(k) ~ k^-4), T_d ~ U[10, 40] K, stars at the centre.

    The Planck-mean opacity model (kappa_model=1) is selected in the params;
    the opacity itself is computed by the method, not here.
    """
    box = box_pc * PC_CM
    lmax, lev, ijk = uniform_structure(n)
    rng = np.random.Generator(np.random.PCG64(seed))
    g = _grf(n, -4.0, rng)
    lnr = math.log(mean_rho) - 0.5 * sigma_ln ** 2 + sigma_ln * g
    rho = np.exp(lnr)
    rho *= mean_rho / rho.mean()
    trng = np.random.Generator(np.random.PCG64(t_seed))
    td = trng.uniform(10.0, 40.0, n ** 3)
    dx = box / n
    if n_stars == 1:
        pos = np.array([[(n // 2 + 0.5) * dx] * 3])
        lum = np.array([star_lum_lsun * LSUN])
    else:
        srng = np.random.Generator(np.random.PCG64(seed + 100))
        pos = srng.uniform(0.25 * box, 0.75 * box, (n_stars, 3))
        lum = np.full(n_stars, star_lum_lsun * LSUN)
    return Workload(name=f"turb{n}", box_cm=box, lmax=lmax, leaf_level=lev, leaf_ijk=ijk,
                    rho=rho.astype(np.float32), td=td.astype(np.float32), star_pos=pos,
                    star_lum=lum, params=default_params(kappa_model=1, **pover), uniform_n=n)


def homogeneous(n: int, box_pc: float, rho0: float, td: float = 20.0, **pover) -> Workload:
    box = box_pc * PC_CM
    lmax, lev, ijk = uniform_structure(n)
    return Workload(name=f"homog{n}", box_cm=box, lmax=lmax, leaf_level=lev, leaf_ijk=ijk,
                    rho=np.full(n ** 3, rho0, np.float32), td=np.full(n ** 3, td, np.float32),
                    params=default_params(**pover), uniform_n=n)


def point_source(n: int = 16, box_pc: float = 0.1, rho0: float = 1e-18, kappa0: float = 0.0,
                 lum_lsun: float = 5.7e4, cell=None, **pover) -> Workload:
    """Point source in a homogeneous medium with dust re-emission switched off."""
    w = homogeneous(n, box_pc, rho0, **pover)
    c = (n // 2, n // 2, n // 2) if cell is None else cell
    dx = w.box_cm / n
    w.star_pos = np.array([[(c[0] + 0.5) * dx, (c[1] + 0.5) * dx, (c[2] + 0.5) * dx]])
    w.star_lum = np.array([lum_lsun * LSUN])
    w.params = default_params(kappa_model=0, kappa0=kappa0, dust_emission=0, **pover)
    w.name = f"point{n}"
    return w


def thick_blob(n: int = 16, box_pc: float = 15.0, r_pc: float = 0.75 * 4, rho_core: float = 1e-17,
               rho_amb: float = 1e-19, t_core: float = 30.0, t_amb: float = 10.0,
               kappa0: float = 5.0, **pover) -> Workload:
    """Isothermal dense blob in a cooler ambient medium (after the thick-blob benchmark)."""
    box = box_pc * PC_CM
    lmax, lev, ijk = uniform_structure(n)
    x = cell_centres(n, box) - 0.5 * box
    r = np.sqrt((x * x).sum(1))
    core = r < r_pc * PC_CM
    rho = np.where(core, rho_core, rho_amb)
    td = np.where(core, t_core, t_amb)
    return Workload(name=f"blob{n}", box_cm=box, lmax=lmax, leaf_level=lev, leaf_ijk=ijk,
                    rho=rho.astype(np.float32), td=td.astype(np.float32),
                    params=default_params(kappa_model=0, kappa0=kappa0, **pover), uniform_n=n)


def random_uniform(n: int, seed: int, box_pc: float = 1.0, thick_frac: float = 0.1,
                   n_stars: int = 2, **pover) -> Workload:
    """Random densities spanning thin and thick cells, random temperatures and stars.

    Used by parity tests to exercise every branch (thin, thick, straddle merges,
    host cells of stars) at sizes the oracle finishes quickly.
    """
    box = box_pc * PC_CM
    lmax, lev, ijk = uniform_structure(n)
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = box / n
    # cell optical depth rho*kappa*dx spans 1e-4 .. 1e2 with kappa0 = 1
    tau = 10.0 ** rng.uniform(-4.0, 0.0, n ** 3)
    thick = rng.uniform(0, 1, n ** 3) < thick_frac
    tau[thick] = 10.0 ** rng.uniform(0.0, 2.0, int(thick.sum()))
    rho = tau / (1.0 * dx)
    td = rng.uniform(8.0, 60.0, n ** 3)
    pos = rng.uniform(0.0, box, (n_stars, 3))
    lum = 10.0 ** rng.uniform(2.0, 5.0, n_stars) * LSUN
    return Workload(name=f"rand{n}s{seed}", box_cm=box, lmax=lmax, leaf_level=lev, leaf_ijk=ijk,
                    rho=rho.astype(np.float32), td=td.astype(np.float32), star_pos=pos,
                    star_lum=lum, params=default_params(kappa_model=0, kappa0=1.0, **pover),
                    uniform_n=n)


def with_gas(w: Workload, seed: int = 7, tgas_lo: float = 10.0, tgas_hi: float = 100.0,
             heat_scale: float = 0.0) -> Workload:
    """Attach a gas temperature (and optionally an extra dust-heating rate) to a workload."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w.tgas = rng.uniform(tgas_lo, tgas_hi, w.n_leaves).astype(np.float32)
    if heat_scale > 0:
        w.heat_extra = (heat_scale * rng.uniform(0.0, 1.0, w.n_leaves)).astype(np.float32)
    return w


def amr_core(n_base_blocks: int = 2, max_level: int = 5, box_pc: float = 0.4,
             m_core_msun: float = 150.0, r_core_pc: float = 0.1, target_leaves: int = 2_000_000,
             seed: int = 4, n_stars: int = 10, perturb: float = 0.2, **pover) -> Workload:
    """AMR octree of 8^3-cell blocks at levels 0..max_level around a collapsing core.

    rho = M / (4 pi R r^2) inside R (so that M(<R) = M), times lognormal
    perturbations exp(perturb*g - perturb^2/2); outside R the density drops to
    the edge value / 100. A block is refined while its peak density exceeds
    c * rho_edge * 4**level; c is bisected so the leaf count lands near
    ``target_leaves``.
    """
    box = box_pc * PC_CM
    R = r_core_pc * PC_CM
    M = m_core_msun * MSUN
    rho_edge = M / (4 * math.pi * R * R * R)
    rng = np.random.Generator(np.random.PCG64(seed))
    lmax = int(round(math.log2(n_base_blocks))) + max_level + 3
    # perturbation field sampled on a coarse periodic lattice and looked up per cell
    gres = 64
    g = _grf(gres, -4.0, rng).reshape(gres, gres, gres)

    def density(cen):
        r = np.sqrt(((cen - 0.5 * box) ** 2).sum(-1))
        r = np.maximum(r, 1e-3 * R)
        base = np.where(r < R, M / (4 * math.pi * R * r * r), rho_edge / 100.0)
        gi = np.clip((cen / box * gres).astype(np.int64), 0, gres - 1)
        pert = np.exp(perturb * g[gi[..., 2], gi[..., 1], gi[..., 0]] - 0.5 * perturb ** 2)
        return base * pert

    def build(cfac):
        lev0 = int(round(math.log2(n_base_blocks)))
        blocks = [(i, j, k, 0) for k in range(n_base_blocks) for j in range(n_base_blocks)
                  for i in range(n_base_blocks)]
        leaves = []
        while blocks:
            nxt = []
            for (bi, bj, bk, bl) in blocks:
                nb = n_base_blocks << bl
                dxb = box / nb
                corner = np.array([bi, bj, bk]) * dxb
                # peak density sampled at the 8^3 cell centres of the block
                cc = (np.indices((8, 8, 8)).reshape(3, -1).T[:, ::-1] + 0.5) * (dxb / 8)
                peak = density(corner + cc).max()
                if bl < max_level and peak > cfac * rho_edge * 4.0 ** bl:
                    for c in range(8):
                        nxt.append((2 * bi + (c & 1), 2 * bj + ((c >> 1) & 1),
                                    2 * bk + ((c >> 2) & 1), bl + 1))
                else:
                    leaves.append((bi, bj, bk, bl + lev0 + 3))
            blocks = nxt
        return leaves

    lo, hi = 1e-3, 1e3
    best = None
    for _ in range(30):
        mid = math.sqrt(lo * hi)
        leaves = build(mid)
        nl = 512 * len(leaves)
        best = (mid, leaves)
        if abs(nl - target_leaves) < 0.05 * target_leaves:
            break
        if nl > target_leaves:
            lo = mid
        else:
            hi = mid
    cfac, leaves = best
    blocks = np.array(leaves, dtype=np.int32)
    nb = blocks.shape[0]
    cell = np.indices((8, 8, 8)).reshape(3, -1).T[:, ::-1].astype(np.int32)  # x fastest
    ijk = (blocks[:, None, :3] * 8 + cell[None, :, :]).reshape(-1, 3).astype(np.int32)
    lev = np.repeat(blocks[:, 3], 512).astype(np.int32)
    lmax = int(lev.max())  # the deepest leaf level actually present
    cen = (ijk.astype(np.float64) + 0.5) * (box / (2.0 ** lev))[:, None]
    rho = density(cen)
    r = np.sqrt(((cen - 0.5 * box) ** 2).sum(-1))
    tgas = np.where(r < R, 20.0, 2000.0)
    srng = np.random.Generator(np.random.PCG64(seed + 1))
    u = srng.standard_normal((n_stars, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    rad = 0.05 * PC_CM * srng.uniform(0, 1, n_stars) ** (1.0 / 3.0)
    pos = 0.5 * box + u * rad[:, None]
    lum = 10.0 ** srng.uniform(2.0, 5.0, n_stars) * LSUN
    w = Workload(name=f"amrcore{nb * 512}", box_cm=box, lmax=lmax, leaf_level=lev, leaf_ijk=ijk,
                 rho=rho.astype(np.float32), td=np.full(rho.shape, 20.0, np.float32),
                 star_pos=pos, star_lum=lum, tgas=tgas.astype(np.float32),
                 params=default_params(kappa_model=1, **pover), blocks=blocks)
    w.params["refine_c"] = cfac
    return w


def amr_random(finest: int, levels: int, seed: int, box_pc: float = 2.0, sigma_ln: float = 1.5,
               refine_frac: float = 0.3, kappa: float = 5.0, **pover) -> Workload:
    """AMR box of 8^3-cell blocks: base grid finest / 2^(levels-1) cells per axis, blocks
    refined (8 children) up to levels-1 times where their peak density is in the top
    refine_frac of their level; density lognormal from a seeded 32^3 Gaussian random field
    (nearest lookup); grey opacity kappa; T_d ~ U[10, 40] K."""
    box = box_pc * PC_CM
    base = finest >> (levels - 1)
    if base < 8 or base % 8:
        raise ValueError("base grid must be a multiple of 8 cells")
    rng = np.random.Generator(np.random.PCG64(seed))
    gres = 32
    g = _grf(gres, -4.0, rng).reshape(gres, gres, gres)
    lb0 = int(round(math.log2(base // 8)))   # block level of the base grid
    def dens(cen):
        gi = np.clip((cen / box * gres).astype(np.int64), 0, gres - 1)
        return np.exp(sigma_ln * g[gi[..., 2], gi[..., 1], gi[..., 0]] - 0.5 * sigma_ln ** 2) * 1e-20
    cc = (np.indices((8, 8, 8)).reshape(3, -1).T[:, ::-1] + 0.5)
    nb0 = base // 8
    blocks = [(i, j, k, 0) for k in range(nb0) for j in range(nb0) for i in range(nb0)]
    leaves = []
    for lev in range(levels):
        if not blocks:
            break
        nbl = nb0 << lev
        dxb = box / nbl
        peaks = np.array([dens(np.array([b[0], b[1], b[2]]) * dxb + cc * (dxb / 8)).max() for b in blocks])
        if lev < levels - 1:
            thr = np.quantile(peaks, 1.0 - refine_frac)
            refine = peaks >= thr
        else:
            refine = np.zeros(len(blocks), bool)
        nxt = []
        for b, r in zip(blocks, refine):
            if r:
                for c in range(8):
                    nxt.append((2 * b[0] + (c & 1), 2 * b[1] + ((c >> 1) & 1), 2 * b[2] + ((c >> 2) & 1), lev + 1))
            else:
                leaves.append((b[0], b[1], b[2], lb0 + lev + 3))
        blocks = nxt
    bl = np.array(leaves, dtype=np.int32)
    cell = np.indices((8, 8, 8)).reshape(3, -1).T[:, ::-1].astype(np.int32)
    ijk = (bl[:, None, :3] * 8 + cell[None, :, :]).reshape(-1, 3).astype(np.int32)
    lev = np.repeat(bl[:, 3], 512).astype(np.int32)
    cen = (ijk.astype(np.float64) + 0.5) * (box / (2.0 ** lev))[:, None]
    rho = dens(cen)
    td = np.random.Generator(np.random.PCG64(seed + 1)).uniform(10.0, 40.0, rho.shape[0])
    return Workload(name=f"amr{finest}L{levels}s{seed}", box_cm=box, lmax=int(lev.max()), leaf_level=lev,
                    leaf_ijk=ijk, rho=rho.astype(np.float32), td=td.astype(np.float32),
                    params=default_params(kappa_model=0, kappa0=kappa, **pover), blocks=bl)


def batch_of_boxes(count: int = 64, seed: int = 5, **pover):
    """Independent boxes of seeded sizes: finest resolution 32, 64 or 128 per axis,
    2 to 5 AMR levels (base grid >= 8 cells), own density seed, grey kappa ~ U[1, 10]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < count:
        finest = int(rng.choice([32, 64, 128]))
        levels = int(rng.integers(2, 6))
        if (finest >> (levels - 1)) < 8:
            continue
        kap = float(rng.uniform(1.0, 10.0))
        out.append(amr_random(finest, levels, seed=int(rng.integers(1 << 30)), kappa=kap, **pover))
    return out


def batch_of_small_boxes(count: int = 512, seed: int = 9, **pover):
    """Many small independent boxes: finest resolution 16 or 32 per axis, 1 or 2 AMR levels
    (base grid >= 8 cells), own density seed, grey kappa ~ U[1, 10] (the batch workload in
    which launch overheads and tails matter)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < count:
        finest = int(rng.choice([16, 32]))
        levels = int(rng.integers(1, 3))
        kap = float(rng.uniform(1.0, 10.0))
        out.append(amr_random(finest, levels, seed=int(rng.integers(1 << 30)), kappa=kap, **pover))
    return out


def batch_of_tiny_boxes(count: int = 1024, seed: int = 10, **pover):
    """Many tiny independent boxes of 8^3 cells (512 targets each, too few to fill the GPU
    in a launch of their own), own density seed, grey kappa ~ U[1, 10]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [amr_random(8, 1, seed=int(rng.integers(1 << 30)), kappa=float(rng.uniform(1.0, 10.0)), **pover)
            for _ in range(count)]


def ionising_field(w: Workload, q_per_lsun: float = 1e44, e_photon_ev: float = 18.0,
                   sigma_d: float = 1.5e-21) -> Workload:
    """Attach a synthetic ionising photon flux and the UV heating it implies.

    phi = sum_s Q_s / (4 pi d_s^2) (unattenuated; the ionising transfer itself is a
    separate module), Q_s = q_per_lsun x L_s / Lsun photons/s; the UV heating
    n_H sigma_d E phi (sigma_d = 1.5e-21 cm^2 per H, mean photon energy 18 eV, n_H =
    0.7 rho / m_H) enters the dust balance as heat_extra.
    """
    n = w.n_leaves
    cen = (w.leaf_ijk.astype(np.float64) + 0.5) * (w.box_cm / (2.0 ** w.leaf_level))[:, None]
    half = 0.5 * w.box_cm / (2.0 ** w.leaf_level)
    phi = np.zeros(n)
    for pos, lum in zip(w.star_pos, w.star_lum):
        d2 = np.maximum(((cen - pos) ** 2).sum(1), half * half)
        phi += q_per_lsun * lum / LSUN / (4 * math.pi * d2)
    nH = 0.7 * w.rho.astype(np.float64) / 1.6726e-24
    w.phi = phi.astype(np.float32)
    w.heat_extra = (nH * sigma_d * e_photon_ev * 1.602e-12 * phi).astype(np.float32)
    return w


def sample_targets(n_leaves: int, count: int, seed: int = 11) -> np.ndarray:
    """Seeded random subset of leaf indices (caller order), sorted, without repeats."""
    rng = np.random.Generator(np.random.PCG64(seed))
    count = min(count, n_leaves)
    return np.sort(rng.choice(n_leaves, size=count, replace=False)).astype(np.int64)


def random_rotations(count: int, seed: int = 13) -> np.ndarray:
    """Seeded uniformly distributed rotations, row-major [count, 3, 3] float64: turned
    orientations of the HEALPix ray set. Unit quaternions from three uniform numbers by
    Shoemake's construction (Graphics Gems III, 1992), then the usual rotation matrix."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u1, u2, u3 = rng.uniform(0.0, 1.0, (3, count))
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    x, y = a * np.sin(2 * math.pi * u2), a * np.cos(2 * math.pi * u2)
    z, w = b * np.sin(2 * math.pi * u3), b * np.cos(2 * math.pi * u3)
    R = np.empty((count, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


BLOB_DIAMETER_PC = {"S": 0.75, "M": 1.5, "L": 3.0}


def blob_suite(variant: str, n: int = 32, **pover) -> Workload:
    """The optically thick blob test: a sphere at 30 K and 1e-17 g/cm^3 in a (15 pc)^3 box
    of 10 K ambient gas at 1e-19 g/cm^3, no background radiation, Planck-mean opacity.
    variant: "S", "M", "L" (diameters 0.75, 1.5, 3 pc); "S-" (S without ambient gas),
    "S+" (S with the ambient density raised tenfold). Grid n^3, blob at the box centre.
    Without ambient gas the ambient cells hold no material at all (density 0)."""
    size = variant[0]
    r_c = 0.5 * BLOB_DIAMETER_PC[size] * PC_CM
    box = 15.0 * PC_CM
    lmax, lev, ijk = uniform_structure(n)
    x = cell_centres(n, box) - 0.5 * box
    r = np.sqrt((x * x).sum(1))
    core = r <= r_c
    rho_a = {"-": 0.0, "+": 1e-18}.get(variant[1:], 1e-19)
    rho = np.where(core, 1e-17, rho_a)
    td = np.where(core, 30.0, 10.0)
    return Workload(name=f"blob{variant}{n}", box_cm=box, lmax=lmax, leaf_level=lev, leaf_ijk=ijk,
                    rho=rho.astype(np.float32), td=td.astype(np.float32),
                    params=default_params(kappa_model=1, **pover), uniform_n=n)
