/*
 * FP64 CPU oracle of the TreeRay/RadPressure hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. The CUDA
 * product path never calls it and shares no code, header, table or constant
 * with it.
 *
 * It follows Klepitko, Walch, Wuensch, Seifried, Dinnbier & Haid (MNRAS 2023),
 * "Tree-based solvers for adaptive mesh refinement code FLASH - III", step by
 * step and in the paper's notation, in plain FP64 with no blocking or fusion:
 *   - grey transfer equation and coefficients a = kappa rho, j = (sigma/pi) kappa rho T^4
 *     (Sec. 2, eqs. rtsimple, alpha) and the Planck-mean opacity model (Sec. 2);
 *   - b-node quantities (Sec. 4.1.1, eqs. lthinbnode, athinbnode, lthickbnode);
 *   - upward propagation and centre of luminosity (Sec. 4.1.2, App. A, eqs.
 *     Lhnodethick..Ahnodethin, COL);
 *   - HEALPix rays, evaluation points, angular kernel alpha and radial kernel beta,
 *     opening criterion (Sec. 4 intro, Sec. 4.2);
 *   - thin and thick mapping (Secs. 4.2.1, 4.2.2, eqs. Lthinmap, Athinmap);
 *   - segment merge, optical depths, extinction and emission (Sec. 4.3, eqs.
 *     tauthin, omegaThick, opt thick, ext inner, fthin, fthick, fcombined,
 *     finalpixelflux);
 *   - ray finalization with J_src (Sec. 4.4, eq. jsrc);
 *   - momentum from flux and trapped source pressure (Sec. 4.5, eqs. psrc,
 *     mom on cell);
 *   - dust thermal balance and radiation temperature (Sec. 4.6, eqs. dust-cool,
 *     dust-heat, radtemp; App. D).
 * Where the paper is silent or ambiguous the reading taken is stated at the
 * function that applies it.
 *
 * Units are CGS. Positions on the tree are integers in units of half a cell of
 * the finest level ("half-units"), so every node centre and every target
 * centre is an integer and all discrete decisions (opening, bin, angular-kernel
 * key) are exact.
 *
 * Parity pins (see tests/test_oracle_*.py): HEALPix round trips and textbook
 * pixel centres; alpha normalisation and antipodal symmetry; the no-extinction
 * brute-force identity J = sum_k L_k / (16 pi^2 r_k^2), also over closest periodic
 * copies; the point-source inverse square law and the paper's extinction fits; the
 * thin-sphere and slab closed forms; zero net flux in an isotropic periodic box; the
 * single-segment limits of App. B; hand-evaluated two-segment extinction; tree moments
 * against direct sums; dust temperature against T_J in the radiative limit and its
 * fixed point; the quarter-turn symmetry of turned HEALPix ray sets; the thick blob's
 * far field (V^(2/3) scaling), plateau and ambient level (Sec. 5.2); the Stroemgren
 * balance of the UV radiation pressure (App. C); values evaluated by hand outside the
 * oracle for J_src, P_src and the escaping S of a star (eqs. jsrc, psrc), the Planck-mean
 * opacity law (Sec. 2), the gas-dust coupling coefficient (App. D) and a segment merge
 * with thick content (Sec. 4.3).
 *
 * Parity unpinned: the readings of the thick path where the paper leaves the choice
 * open (the full A~ of every thick node touching a ray segment, the blend of thin and
 * thick flux when neither weighs) are pinned only through their limits (deep-thick
 * plateau, compact thick body, blob far field and plateau) and the merge through one
 * hand-evaluated case, not against an independent transfer solution.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* physical constants, CGS */
#define OR_PI 3.14159265358979323846
#define OR_SIGMA 5.670374419e-5  /* Stefan-Boltzmann */
#define OR_C 2.99792458e10        /* speed of light */
#define OR_MH 1.6726e-24          /* hydrogen mass */
#define OR_XH 0.7                 /* hydrogen mass fraction */
#define OR_TFLOOR 2.7             /* dust temperature floor, Sec. 4.6 */

/* ------------------------------------------------------------------ params */

typedef struct {
    int npix;              /* 12 * nside^2 HEALPix rays */
    int nbins;             /* radial evaluation points per ray */
    double theta;          /* opening angle theta_lim; < 0: sqrt(4 pi / npix), ray-matched */
    int kappa_model;       /* 0: grey kappa0, 1: Planck mean 0.1 (T/10K)^2, capped at 150 K */
    double kappa0;         /* grey opacity per gram of gas */
    double dust_to_gas;    /* xi; enters only the gas-dust coupling */
    int dust_emission;     /* 0 switches dust re-emission off (point-source benchmark) */
    double kappa_ext_scale;/* scales the extinction areas A~ (test switch) */
    int alpha_s;           /* sub-points per axis of the angular kernel's sampling */
    int periodic;          /* bit a set: axis a is periodic (nearest copies, Sec. 4.2) */
    int bin_spacing;       /* 0: geometric radii, 1: quadratically growing radii (Sec. 4.2) */
    int col_mapping;       /* 1: map accepted nodes at their centre of luminosity (Sec. 7.6) */
} or_params;

/* ------------------------------------------------------------------ HEALPix
 * Nested-scheme pixelisation of Gorski et al. (2005, ApJ 622, 759): 12 base
 * faces, each split into nside x nside pixels whose (ix, iy) bits are
 * interleaved. The steps (polar caps against the equatorial belt, the face
 * index from the two edge indices, the ring shift, and the base-face row and
 * column tables) are those of the standard published algorithm, as the HEALPix
 * library's nested ang2pix / pix2vec implement it; the names here are the
 * paper's symbols. */

static const int or_jrll[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
static const int or_jpll[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

static int64_t or_interleave(int64_t ix, int64_t iy) {
    int64_t p = 0;
    for (int b = 0; b < 30; ++b) {
        p |= ((ix >> b) & 1) << (2 * b);
        p |= ((iy >> b) & 1) << (2 * b + 1);
    }
    return p;
}

static void or_deinterleave(int64_t p, int64_t* ix, int64_t* iy) {
    int64_t x = 0, y = 0;
    for (int b = 0; b < 30; ++b) {
        x |= ((p >> (2 * b)) & 1) << b;
        y |= ((p >> (2 * b + 1)) & 1) << b;
    }
    *ix = x;
    *iy = y;
}

/* Direction (x, y, z), not necessarily normalised, to nested pixel index. */
int or_ang2pix(int nside, double x, double y, double z) {
    double r2 = x * x + y * y + z * z;
    double r = sqrt(r2);
    double cz = z / r;
    double za = fabs(cz);
    double phi = atan2(y, x);
    if (phi < 0.0) phi += 2.0 * OR_PI;
    double tt = phi * (2.0 / OR_PI);
    if (tt >= 4.0) tt -= 4.0;
    int64_t ns = nside, face, ix, iy;
    if (za <= 2.0 / 3.0) {
        double t1 = (double)ns * (0.5 + tt);
        double t2 = (double)ns * (cz * 0.75);
        int64_t jp = (int64_t)(t1 - t2);
        int64_t jm = (int64_t)(t1 + t2);
        int64_t ifp = jp / ns, ifm = jm / ns;
        if (ifp == ifm) face = ifp | 4;
        else if (ifp < ifm) face = ifp;
        else face = ifm + 8;
        ix = jm & (ns - 1);
        iy = ns - (jp & (ns - 1)) - 1;
    } else {
        int64_t ntt = (int64_t)tt;
        if (ntt > 3) ntt = 3;
        double tp = tt - (double)ntt;
        /* 3 (1 - |z|/r) evaluated without cancellation as 3 (x^2+y^2) / (r (r + |z|)) */
        double omz = 3.0 * ((x * x + y * y) / (r * (r + fabs(z))));
        double tmp = (double)ns * sqrt(omz);
        int64_t jp = (int64_t)(tp * tmp);
        int64_t jm = (int64_t)((1.0 - tp) * tmp);
        if (jp > ns - 1) jp = ns - 1;
        if (jm > ns - 1) jm = ns - 1;
        if (cz >= 0) {
            face = ntt;
            ix = ns - jm - 1;
            iy = ns - jp - 1;
        } else {
            face = ntt + 8;
            ix = jp;
            iy = jm;
        }
    }
    return (int)(face * ns * ns + or_interleave(ix, iy));
}

/* Nested pixel index to the unit vector of its centre. */
void or_pix2vec(int nside, int pix, double* v) {
    int64_t ns = nside, npface = ns * ns;
    int64_t face = pix / npface, ix, iy;
    or_deinterleave(pix % npface, &ix, &iy);
    int64_t jr = or_jrll[face] * ns - (ix + iy) - 1;
    int64_t nr, kshift;
    double z;
    if (jr < ns) {
        nr = jr;
        z = 1.0 - (double)(nr * nr) / (3.0 * (double)npface);
        kshift = 0;
    } else if (jr > 3 * ns) {
        nr = 4 * ns - jr;
        z = -(1.0 - (double)(nr * nr) / (3.0 * (double)npface));
        kshift = 0;
    } else {
        nr = ns;
        z = (double)(2 * ns - jr) * 2.0 / (3.0 * (double)ns);
        kshift = (jr - ns) & 1;
    }
    int64_t jp = (or_jpll[face] * nr + ix - iy + 1 + kshift) / 2;
    if (jp > 4 * ns) jp -= 4 * ns;
    if (jp < 1) jp += 4 * ns;
    double phi = ((double)jp - 0.5 * (double)(kshift + 1)) * (OR_PI / 2.0) / (double)nr;
    double st = sqrt((1.0 - z) * (1.0 + z));
    v[0] = st * cos(phi);
    v[1] = st * sin(phi);
    v[2] = z;
}

static int or_nside(int npix) {
    int ns = 1;
    while (12 * ns * ns < npix) ns *= 2;
    return (12 * ns * ns == npix) ? ns : -1;
}

/* --------------------------------------------------------- angular kernel
 * alpha_node(h): fraction of the node's volume whose direction from the target
 * falls into ray h. The paper tabulates Monte-Carlo overlap fractions on discrete
 * node positions (Sec. 4.2). Reading: the position is the node-centre offset o
 * from the target in units of 1/8 of the node edge E, K = 8 o / E, kept exact when
 * integral and otherwise replaced by the nearest odd integer; the node cube is
 * sampled on an s x s x s lattice of sub-cube centres, which as seen from the
 * target lie along the integer vectors 2K + 2a - 7 (s = 8). The target's own cell
 * (o = 0) gets 1/N_pix on every ray. */

static void or_key(const int64_t* o, int64_t E, int64_t* K) {
    for (int a = 0; a < 3; ++a) {
        int64_t num = 8 * o[a];
        if (num % E == 0) {
            K[a] = num / E;
        } else {
            /* floor(4 o / E) for either sign */
            int64_t q = (4 * o[a]) / E;
            if ((4 * o[a]) % E != 0 && o[a] < 0) q -= 1;
            K[a] = 2 * q + 1;
        }
    }
}

/* Hit counts of the s^3 sample directions per pixel for key K. counts: int[npix].
 * rot (may be NULL): the ray set of a turned HEALPix orientation (Sec. 7.6), a row-major
 * rotation R; ray h of that orientation points along R n_h, so a sample direction v is
 * counted in ray h when R^T v lies in pixel h. (R^T v)_a = R_0a v_x + R_1a v_y + R_2a v_z,
 * summed in that order. */
void or_alpha_counts_rot(int npix, int s, const int64_t* K, const double* rot, int* counts) {
    int nside = or_nside(npix);
    memset(counts, 0, sizeof(int) * npix);
    for (int c = 0; c < s; ++c)
        for (int b = 0; b < s; ++b)
            for (int a = 0; a < s; ++a) {
                /* sample centre ((a + 1/2)/s - 1/2) E from the node centre, in units E/(2s) */
                double vx = (double)(2 * s * K[0] / 8 + 2 * a + 1 - s);
                double vy = (double)(2 * s * K[1] / 8 + 2 * b + 1 - s);
                double vz = (double)(2 * s * K[2] / 8 + 2 * c + 1 - s);
                if (rot) {
                    double wx = rot[0] * vx + rot[3] * vy + rot[6] * vz;
                    double wy = rot[1] * vx + rot[4] * vy + rot[7] * vz;
                    double wz = rot[2] * vx + rot[5] * vy + rot[8] * vz;
                    vx = wx;
                    vy = wy;
                    vz = wz;
                }
                counts[or_ang2pix(nside, vx, vy, vz)]++;
            }
}

void or_alpha_counts(int npix, int s, const int64_t* K, int* counts) {
    or_alpha_counts_rot(npix, s, K, NULL, counts);
}

/* Lazily filled alpha cache: open-addressing hash table of fixed capacity,
 * filled concurrently with compare-and-swap. A full table (never expected at
 * the sizes used) falls back to computing the list for every call. */
#define OR_HCAP (1 << 21)
typedef struct {
    int npix, s, D;
    uint64_t* keys;   /* packed key + 1, 0 = empty */
    int** lists;      /* per slot: pairs (pixel, count), terminated by -1 */
    const double* rot;/* orientation of the ray set (NULL: the unturned HEALPix grid) */
} or_alpha_table;

static uint64_t or_pack(const int64_t* K) {
    return ((uint64_t)(K[0] + (1 << 20))) | ((uint64_t)(K[1] + (1 << 20)) << 21) |
           ((uint64_t)(K[2] + (1 << 20)) << 42);
}

static int* or_alpha_make(const or_alpha_table* t, const int64_t* K) {
    int* counts = (int*)malloc(sizeof(int) * t->npix);
    or_alpha_counts_rot(t->npix, t->s, K, t->rot, counts);
    int n = 0;
    for (int h = 0; h < t->npix; ++h) n += counts[h] > 0;
    int* out = (int*)malloc(sizeof(int) * (2 * n + 1));
    int j = 0;
    for (int h = 0; h < t->npix; ++h)
        if (counts[h] > 0) {
            out[j++] = h;
            out[j++] = counts[h];
        }
    out[j] = -1;
    free(counts);
    return out;
}

/* Pixel/count list of key K; *owned = 1 when the caller must free it. */
static const int* or_alpha_get(or_alpha_table* t, const int64_t* K, int* owned) {
    uint64_t pk = or_pack(K) + 1;
    uint64_t h = (pk * 0x9E3779B97F4A7C15ull) >> 43;
    *owned = 0;
    for (int probe = 0; probe < 4096; ++probe) {
        uint64_t slot = (h + (uint64_t)probe) & (OR_HCAP - 1);
        uint64_t cur = __atomic_load_n(&t->keys[slot], __ATOMIC_ACQUIRE);
        if (cur == 0) {
            uint64_t expect = 0;
            if (__atomic_compare_exchange_n(&t->keys[slot], &expect, pk, 0, __ATOMIC_ACQ_REL,
                                            __ATOMIC_ACQUIRE)) {
                int* l = or_alpha_make(t, K);
                __atomic_store_n(&t->lists[slot], l, __ATOMIC_RELEASE);
                return l;
            }
            cur = expect;
        }
        if (cur == pk) {
            int* l;
            while ((l = __atomic_load_n(&t->lists[slot], __ATOMIC_ACQUIRE)) == NULL) {
            }
            return l;
        }
    }
    *owned = 1;
    return or_alpha_make(t, K);
}

/* -------------------------------------------------------------------- tree */

typedef struct {
    int level;
    int leaf;             /* caller index of the leaf, -1 for h-nodes */
    int child[8];         /* node ids of the sub-nodes, Morton child order x|y<<1|z<<2 */
    int64_t c[3];         /* geometric centre, half-units */
    int64_t E;            /* edge, half-units */
    uint64_t prefix;      /* Morton prefix at its level */
    /* thin and thick sums (Sec. 4.1, App. A) */
    double Lt, At, Vt;    /* thin luminosity (+S), area A~, volume */
    double LVk, Ak, Vk;   /* thick: sum of L_ (per area per sr) x V, area A~, volume */
    double m;             /* mass */
    double xi;            /* this node's own COL weight as a sub-node */
    double col[3];        /* centre of luminosity, half-units (absolute) */
    int thick;            /* leaves: tau_b >= 1 */
} or_node;

typedef struct {
    or_params p;
    int lmax;
    double box, u;        /* box edge (cm), half-unit (cm) */
    int64_t nleaves, nnodes;
    or_node* nodes;       /* level-major, Morton order inside a level (breadth first) */
    int* leaf_node;       /* caller leaf index -> node id */
    int* leaf_level;
    double* kap;          /* per leaf opacity */
    double* tau;          /* per leaf tau_b */
    double* Jsrc;         /* per leaf J_src,IR */
    double* Psrc;         /* per leaf P_src */
    double* rho;
    or_alpha_table alpha;
    int level_first[64], level_count[64];
    /* several HEALPix orientations (Sec. 7.6); n_orient = 0: the single unturned one */
    int n_orient;
    double* rot;            /* [n_orient][9] row-major rotations R_o */
    uint8_t* orient;        /* per leaf: its orientation (caller leaf index) */
    or_alpha_table* oalpha; /* [n_orient] angular kernels of the turned ray sets */
} or_tree;

static uint64_t or_morton(uint64_t x, uint64_t y, uint64_t z, int bits) {
    uint64_t k = 0;
    for (int b = 0; b < bits; ++b) {
        k |= ((x >> b) & 1ull) << (3 * b);
        k |= ((y >> b) & 1ull) << (3 * b + 1);
        k |= ((z >> b) & 1ull) << (3 * b + 2);
    }
    return k;
}

typedef struct {
    uint64_t key;  /* Morton key of the leaf's lower corner at the finest level */
    int id;
} or_kv;

static int or_kv_cmp(const void* a, const void* b) {
    uint64_t x = ((const or_kv*)a)->key, y = ((const or_kv*)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}

typedef struct {
    or_kv* kv;
    const int32_t* lev;
    int lmax;
    or_node* tmp;
    int64_t ntmp, cap;
    int err;
} or_builder;

/* Recursive octree construction over the Morton-sorted leaves [lo, hi) that lie
 * inside the node (level, prefix). Returns the temporary node id. */
static int64_t or_build_rec(or_builder* b, int level, uint64_t prefix, int64_t lo, int64_t hi) {
    if (hi <= lo || b->err) {
        b->err = 1;
        return -1;
    }
    if (b->ntmp == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 1024;
        b->tmp = (or_node*)realloc(b->tmp, sizeof(or_node) * b->cap);
    }
    int64_t id = b->ntmp++;
    or_node nd;
    memset(&nd, 0, sizeof(nd));
    nd.level = level;
    nd.prefix = prefix;
    nd.leaf = -1;
    for (int k = 0; k < 8; ++k) nd.child[k] = -1;
    int shift = 3 * (b->lmax - level);
    if (hi - lo == 1 && b->lev[b->kv[lo].id] == level) {
        nd.leaf = b->kv[lo].id;
        b->tmp[id] = nd;
        return id;
    }
    if (level >= b->lmax) {
        b->err = 2;
        b->tmp[id] = nd;
        return id;
    }
    b->tmp[id] = nd;
    int64_t start = lo;
    for (int k = 0; k < 8; ++k) {
        uint64_t cp = (prefix << 3) | (uint64_t)k;
        int cshift = shift - 3;
        int64_t end = start;
        while (end < hi && (b->kv[end].key >> cshift) == cp) ++end;
        int64_t cid = or_build_rec(b, level + 1, cp, start, end);
        b->tmp[id].child[k] = (int)cid;
        start = end;
    }
    if (start != hi) b->err = 3;
    return id;
}

static double or_kappa(const or_params* p, double T, const float* kin, int64_t k) {
    if (kin) return (double)kin[k];
    if (p->kappa_model == 0) return p->kappa0;
    double Tc = T < 150.0 ? T : 150.0;
    return 1.0e-3 * (Tc * Tc); /* 0.1 cm^2/g x (T / 10 K)^2, Sec. 2 */
}

static void or_alpha_free(or_alpha_table* a) {
    if (a->lists) {
        for (int64_t i = 0; i < OR_HCAP; ++i) free(a->lists[i]);
        free(a->lists);
        free(a->keys);
    }
    a->lists = NULL;
    a->keys = NULL;
}

static void or_orient_free(or_tree* t) {
    for (int o = 0; o < t->n_orient; ++o) or_alpha_free(&t->oalpha[o]);
    free(t->oalpha);
    free(t->rot);
    free(t->orient);
    t->oalpha = NULL;
    t->rot = NULL;
    t->orient = NULL;
    t->n_orient = 0;
}

void or_tree_free(or_tree* t) {
    if (!t) return;
    or_alpha_free(&t->alpha);
    or_orient_free(t);
    free(t->nodes);
    free(t->leaf_node);
    free(t->leaf_level);
    free(t->kap);
    free(t->tau);
    free(t->Jsrc);
    free(t->Psrc);
    free(t->rho);
    free(t);
}

/*
 * Tree build (Sec. 4.1): b-node quantities, then upward sums and COL (App. A).
 *
 * Readings where the paper is silent:
 *  - S (point sources) of every b-node, thin or thick, goes into the thin
 *    luminosity channel (the "+S" of eq. Lhnodethin).
 *  - Thick h-node luminosity is propagated as sum L_ V (volume-weighted), so that
 *    the thick mapping, which multiplies by V_node, is exact for b-nodes.
 *  - The COL of an h-node weights the sub-nodes' own COLs (b-nodes: their centres);
 *    an h-node sub-node's weight is xi = L_thin + (sum L_ V / V_thick) V_thick^(2/3).
 *  - A star heats the b-node that contains its position (half-open cells).
 * Sums run over sub-nodes in Morton child order from 0.0, without contraction.
 */
int or_build(const or_params* p, int lmax, double box_cm, int64_t nleaves,
             const int32_t* leaf_level, const int32_t* leaf_ijk, const float* rho,
             const float* Td, const float* kappa_in, int nstars, const double* star_pos,
             const double* star_L, or_tree** out) {
    *out = NULL;
    if (nleaves <= 0 || lmax < 0 || lmax > 19 || or_nside(p->npix) < 0 || p->nbins < 1 ||
        p->nbins > 64)
        return 1;
    or_tree* t = (or_tree*)calloc(1, sizeof(or_tree));
    t->p = *p;
    /* theta < 0: the opening angle matched to the ray size, sqrt(4 pi / N_pix)
     * (Sec. 7.6: more rays open nodes further, toward the ray's angular size) */
    if (t->p.theta < 0.0) t->p.theta = sqrt(4.0 * OR_PI / (double)p->npix);
    t->lmax = lmax;
    t->box = box_cm;
    t->u = ldexp(box_cm, -(lmax + 1));
    t->nleaves = nleaves;

    /* Morton-sort the leaves by their lower-corner key at the finest level */
    or_kv* kv = (or_kv*)malloc(sizeof(or_kv) * nleaves);
    for (int64_t k = 0; k < nleaves; ++k) {
        int l = leaf_level[k];
        uint64_t sh = (uint64_t)(lmax - l);
        kv[k].key = or_morton((uint64_t)leaf_ijk[3 * k] << sh, (uint64_t)leaf_ijk[3 * k + 1] << sh,
                              (uint64_t)leaf_ijk[3 * k + 2] << sh, lmax);
        kv[k].id = (int)k;
    }
    qsort(kv, nleaves, sizeof(or_kv), or_kv_cmp);
    or_builder b = {kv, leaf_level, lmax, NULL, 0, 0, 0};
    or_build_rec(&b, 0, 0, 0, nleaves);
    free(kv);
    if (b.err) {
        free(b.tmp);
        free(t);
        return 2;
    }

    /* breadth-first renumbering: level-major, Morton order within a level */
    int64_t nn = b.ntmp;
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * nn);
    int64_t* newid = (int64_t*)malloc(sizeof(int64_t) * nn);
    int64_t head = 0, tail = 0;
    order[tail++] = 0;
    while (head < tail) {
        int64_t id = order[head++];
        for (int k = 0; k < 8; ++k)
            if (b.tmp[id].child[k] >= 0) order[tail++] = b.tmp[id].child[k];
    }
    for (int64_t i = 0; i < nn; ++i) newid[order[i]] = i;
    t->nnodes = nn;
    t->nodes = (or_node*)calloc(nn, sizeof(or_node));
    for (int64_t i = 0; i < nn; ++i) {
        or_node nd = b.tmp[order[i]];
        for (int k = 0; k < 8; ++k)
            if (nd.child[k] >= 0) nd.child[k] = (int)newid[nd.child[k]];
        t->nodes[i] = nd;
    }
    free(order);
    free(newid);
    free(b.tmp);
    for (int l = 0; l < 64; ++l) t->level_first[l] = -1, t->level_count[l] = 0;
    for (int64_t i = 0; i < nn; ++i) {
        int l = t->nodes[i].level;
        if (t->level_first[l] < 0) t->level_first[l] = (int)i;
        t->level_count[l]++;
    }

    /* geometry in half-units */
    for (int64_t i = 0; i < nn; ++i) {
        or_node* nd = &t->nodes[i];
        int l = nd->level;
        nd->E = (int64_t)2 << (lmax - l);
        uint64_t a = 0, bb = 0, c = 0;
        for (int bit = 0; bit < l; ++bit) {
            a |= ((nd->prefix >> (3 * bit)) & 1ull) << bit;
            bb |= ((nd->prefix >> (3 * bit + 1)) & 1ull) << bit;
            c |= ((nd->prefix >> (3 * bit + 2)) & 1ull) << bit;
        }
        nd->c[0] = (2 * (int64_t)a + 1) * (nd->E / 2);
        nd->c[1] = (2 * (int64_t)bb + 1) * (nd->E / 2);
        nd->c[2] = (2 * (int64_t)c + 1) * (nd->E / 2);
    }

    /* b-node quantities (Sec. 4.1.1) */
    t->leaf_node = (int*)malloc(sizeof(int) * nleaves);
    t->leaf_level = (int*)malloc(sizeof(int) * nleaves);
    t->kap = (double*)malloc(sizeof(double) * nleaves);
    t->tau = (double*)malloc(sizeof(double) * nleaves);
    t->Jsrc = (double*)calloc(nleaves, sizeof(double));
    t->Psrc = (double*)calloc(nleaves, sizeof(double));
    t->rho = (double*)malloc(sizeof(double) * nleaves);
    for (int64_t i = 0; i < nn; ++i)
        if (t->nodes[i].leaf >= 0) t->leaf_node[t->nodes[i].leaf] = (int)i;

    /* luminosity of the stars hosted by each leaf, summed in input order */
    double* Lsrc = (double*)calloc(nleaves, sizeof(double));
    double dxf = ldexp(box_cm, -lmax);
    for (int s = 0; s < nstars; ++s) {
        int64_t f[3];
        for (int a = 0; a < 3; ++a) {
            double q = floor(star_pos[3 * s + a] / dxf);
            int64_t fi = (int64_t)q;
            if (q < 0) fi = 0;
            if (q > (double)(((int64_t)1 << lmax) - 1)) fi = ((int64_t)1 << lmax) - 1;
            f[a] = fi;
        }
        /* descend from the root to the leaf containing finest cell f */
        int64_t id = 0;
        while (t->nodes[id].leaf < 0) {
            int l = t->nodes[id].level;
            int sh = lmax - l - 1;
            int k = (int)(((f[0] >> sh) & 1) | (((f[1] >> sh) & 1) << 1) | (((f[2] >> sh) & 1) << 2));
            id = t->nodes[id].child[k];
        }
        Lsrc[t->nodes[id].leaf] += star_L[s];
    }

    const double sig_pi = OR_SIGMA / OR_PI;
    for (int64_t k = 0; k < nleaves; ++k) {
        or_node* nd = &t->nodes[t->leaf_node[k]];
        int l = leaf_level[k];
        double T = (double)Td[k];
        double rh = (double)rho[k];
        double kap = or_kappa(p, T, kappa_in, k);
        double dx = ldexp(box_cm, -l);
        double dV = (dx * dx) * dx;
        double rk = rh * kap;
        double tau = rk * dx;                       /* tau_b-node = rho kappa dr */
        int thick = tau >= 1.0;                     /* thin iff tau_b < 1 */
        double T4 = (T * T) * (T * T);
        double A = (rk * dV) * p->kappa_ext_scale;  /* A~ = rho kappa dV, eq. athinbnode */
        double ext = exp(-0.5 * tau);
        double S = Lsrc[k] * ext;                   /* S = L_src,IR e^(-tau_b/2) */
        t->kap[k] = kap;
        t->tau[k] = tau;
        t->rho[k] = rh;
        t->leaf_level[k] = l;
        t->Jsrc[k] = ((1.0 - ext) * Lsrc[k]) / (dx * dx);          /* eq. jsrc, V_src = V_b */
        t->Psrc[k] = ((1.0 - ext) * Lsrc[k]) / (OR_C * (dx * dx)); /* eq. psrc, A_src = dx^2 */
        nd->thick = thick;
        nd->m = rh * dV;
        if (!thick) {
            double L = p->dust_emission ? (((4.0 * OR_SIGMA) * rk) * T4) * dV : 0.0; /* eq. lthinbnode */
            nd->Lt = L + S;
            nd->At = A;
            nd->Vt = dV;
            nd->LVk = nd->Ak = nd->Vk = 0.0;
            nd->xi = nd->Lt;
        } else {
            double Lu = p->dust_emission ? sig_pi * T4 : 0.0; /* eq. lthickbnode */
            nd->Lt = S;
            nd->At = 0.0;
            nd->Vt = 0.0;
            nd->LVk = Lu * dV;
            nd->Ak = A;
            nd->Vk = dV;
            nd->xi = S + Lu * (dx * dx); /* L_ V^(2/3) plus the source */
        }
        for (int a = 0; a < 3; ++a) nd->col[a] = (double)nd->c[a];
    }
    free(Lsrc);

    /* upward propagation (App. A), deepest level first */
    for (int l = lmax - 1; l >= 0; --l) {
        if (t->level_first[l] < 0) continue;
        for (int64_t i = t->level_first[l]; i < t->level_first[l] + t->level_count[l]; ++i) {
            or_node* nd = &t->nodes[i];
            if (nd->leaf >= 0) continue;
            double Lt = 0.0, At = 0.0, Vt = 0.0, LVk = 0.0, Ak = 0.0, Vk = 0.0, m = 0.0;
            double Xi = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
            for (int k = 0; k < 8; ++k) {
                const or_node* ch = &t->nodes[nd->child[k]];
                Lt = Lt + ch->Lt;
                At = At + ch->At;
                Vt = Vt + ch->Vt;
                LVk = LVk + ch->LVk;
                Ak = Ak + ch->Ak;
                Vk = Vk + ch->Vk;
                m = m + ch->m;
                Xi = Xi + ch->xi;
                cx = cx + ch->xi * ch->col[0];
                cy = cy + ch->xi * ch->col[1];
                cz = cz + ch->xi * ch->col[2];
            }
            nd->Lt = Lt;
            nd->At = At;
            nd->Vt = Vt;
            nd->LVk = LVk;
            nd->Ak = Ak;
            nd->Vk = Vk;
            nd->m = m;
            if (Vk > 0.0) {
                double cb = cbrt(Vk);
                nd->xi = Lt + (LVk / Vk) * (cb * cb);
            } else {
                nd->xi = Lt;
            }
            if (Xi > 0.0) {
                nd->col[0] = cx / Xi;
                nd->col[1] = cy / Xi;
                nd->col[2] = cz / Xi;
            } else {
                for (int a = 0; a < 3; ++a) nd->col[a] = (double)nd->c[a];
            }
        }
    }

    t->alpha.npix = p->npix;
    t->alpha.s = p->alpha_s;
    t->alpha.keys = (uint64_t*)calloc(OR_HCAP, sizeof(uint64_t));
    t->alpha.lists = (int**)calloc(OR_HCAP, sizeof(int*));
    *out = t;
    return 0;
}

/* ------------------------------------------------------------- evaluation */

/* Evaluation points R_i (half-units) of a target of edge Et (Sec. 4.2, Fig. ray bin).
 * Reading: R_0 = Et / 2 (half the target cell), R_i = R_0 (R_max / R_0)^(i / N) with
 * R_max = sqrt(3) x box edge (geometric spacing). Segment i is [R_i, R_(i+1)); segment
 * 0 also holds [0, R_0); nodes beyond R_(N-1) fall into the last segment. */
static void or_radii(int nbins, int lmax, int periodic, int spacing, int64_t Et, double* R) {
    double R0 = 0.5 * (double)Et;
    double B = (double)((int64_t)2 << lmax);
    double Rmax = sqrt(3.0) * B;
    if (periodic) { /* largest nearest-copy distance: half the box on periodic axes */
        double s = 0.0;
        for (int a = 0; a < 3; ++a) {
            double e = ((periodic >> a) & 1) ? 0.5 * B : B;
            s += e * e;
        }
        Rmax = sqrt(s);
    }
    if (spacing == 1) { /* radii growing quadratically from R_0 to R_max */
        for (int i = 0; i <= nbins; ++i) {
            double q = (double)i / (double)nbins;
            R[i] = R0 + (Rmax - R0) * (q * q);
        }
        return;
    }
    for (int i = 0; i <= nbins; ++i) R[i] = R0 * pow(Rmax / R0, (double)i / (double)nbins);
}

/* Offset from the target to the closest periodic copy of a node (Sec. 4.2: "only the
 * closest ones are considered"): on a periodic axis the offset is brought into
 * [-B/2, B/2], B the box edge in half-units. An offset of exactly B/2 has two closest
 * copies, at +B/2 and -B/2; the returned mask marks those axes (reading: both copies
 * count, each with weight 1/2 per such axis). */
static int or_nearest(const or_tree* t, const or_node* nd, const or_node* tn, int64_t* o) {
    int64_t B = (int64_t)2 << t->lmax, half = B / 2;
    int ties = 0;
    for (int a = 0; a < 3; ++a) {
        o[a] = nd->c[a] - tn->c[a];
        if ((t->p.periodic >> a) & 1) {
            if (o[a] > half) o[a] -= B;
            else if (o[a] < -half) o[a] += B;
            if (o[a] == half || o[a] == -half) ties |= 1 << a;
        }
    }
    return ties;
}

static int or_bin(int nbins, const double* R, double d2) {
    int i = 0;
    for (int j = 1; j < nbins; ++j)
        if (d2 >= R[j] * R[j]) i = j;
    return i;
}

typedef struct {
    int npix, nbins;
    double *Lth, *Ath, *Lk, *Ak, *Vk, *Qk; /* [nbins][npix] */
    uint64_t* flag;                        /* [npix]: bit i = thick material spans i, i+1 */
} or_rays;

/*
 * Mapping of one accepted node onto the rays (Secs. 4.2.1, 4.2.2).
 *   beta = R_i^2 / r^2 with r the distance from the target to the node's COL
 *     (reading: eq. for beta prints the inverse, but the text requires that the
 *     flux of beta L at R_i equals that of L at r; exact beta* is used);
 *     beta = 1 for the target's own cell.
 *   thin:  L^ += alpha beta L,  A^ += alpha beta A~
 *   thick: L^ += alpha L_ V,    A^ += A~ (every ray the node touches),
 *          V^ += alpha V,       Q^ += alpha beta V
 * Thick material whose radial extent [d - sqrt3/2 E, d + sqrt3/2 E] crosses
 * segment boundaries flags those boundaries for merging (Sec. 4.3).
 * w: weight of this copy of the node (1, or 1/2 per axis with two closest copies).
 */
static void or_map_node(const or_tree* t, or_alpha_table* at, const or_node* nd, const int64_t* o,
                        int64_t d2, const double* R, or_rays* ry, double w) {
    int nb = ry->nbins, np = ry->npix;
    double u = t->u;
    int own = (d2 == 0);
    /* mapping at the centre of luminosity (Sec. 7.6: the nodes are shifted towards their
     * centre of emission when they are mapped to rays), for nodes whose COL is off centre.
     * Reading: every mapping decision is taken at the COL position p = o + (COL - centre)
     * instead of the centre, in FP64: the segment is the largest j with |p|^2 >= R_j^2, the
     * straddled boundaries compare |p|^2 with (R_j +- s)^2, and the angular key is the odd
     * grid point 2 floor(4 p / E) + 1 per axis (p is no grid point, so K = 8 o / E cannot
     * be integral); |p|^2 = (p_x^2 + p_y^2) + p_z^2. The opening test stays at the centre. */
    double pc[3] = {0.0, 0.0, 0.0}, pd2 = 0.0;
    int colmap = 0;
    if (t->p.col_mapping && !own) {
        for (int a = 0; a < 3; ++a) {
            double c = nd->col[a] - (double)nd->c[a];
            if (c != 0.0) colmap = 1;
            pc[a] = (double)o[a] + c;
        }
        pd2 = (pc[0] * pc[0] + pc[1] * pc[1]) + pc[2] * pc[2];
    }
    int i = or_bin(nb, R, colmap ? pd2 : (double)d2);
    double beta = 1.0;
    if (!own) {
        double r2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double q = (double)o[a] + (nd->col[a] - (double)nd->c[a]);
            r2 += q * q;
        }
        beta = (R[i] * R[i]) / r2;
    }
    int64_t K[3] = {0, 0, 0};
    const int* lst = NULL;
    int owned = 0;
    if (!own) {
        if (colmap) {
            for (int a = 0; a < 3; ++a) K[a] = 2 * (int64_t)floor(4.0 * pc[a] / (double)nd->E) + 1;
        } else {
            or_key(o, nd->E, K);
        }
        lst = or_alpha_get(at, K, &owned);
    }
    int ilo = 0, ihi = 0;
    if (nd->Vk > 0.0) {
        double s = (sqrt(3.0) * 0.5) * (double)nd->E;
        for (int j = 1; j < nb; ++j) {
            double up = R[j] + s;
            double dn = R[j] - s;
            double x2 = colmap ? pd2 : (double)d2;
            if (x2 >= up * up) ilo = j;
            if (dn <= 0.0 || x2 >= dn * dn) ihi = j;
        }
    }
    /* values in CGS: luminosities erg/s, areas cm^2, volumes cm^3; w < 1 for one of
     * several closest periodic copies */
    double Lt = w * nd->Lt, At = w * nd->At, LVk = w * nd->LVk, Ak = w * nd->Ak, Vk = w * nd->Vk;
    (void)u;
    int n = own ? np : 0;
    if (!own)
        while (lst[2 * n] >= 0) ++n;
    for (int e = 0; e < n; ++e) {
        int h = own ? e : lst[2 * e];
        double a = own ? 1.0 / (double)np : (double)lst[2 * e + 1] / (double)(t->p.alpha_s * t->p.alpha_s * t->p.alpha_s);
        int64_t c = (int64_t)i * np + h;
        ry->Lth[c] += a * beta * Lt;
        ry->Ath[c] += a * beta * At;
        if (Vk > 0.0) {
            ry->Lk[c] += a * LVk;
            ry->Ak[c] += Ak;
            ry->Vk[c] += a * Vk;
            ry->Qk[c] += a * beta * Vk;
            for (int j = ilo; j < ihi; ++j) ry->flag[h] |= 1ull << j;
        }
    }
    if (owned) free((void*)lst);
}

/*
 * Integration of one ray from the inside out (Sec. 4.3) in CGS.
 * Inputs per segment i (already in CGS): Lth, Ath, Lk, Ak, Vk, Qk, radii R (cm),
 * merge flags. Returns the flux F received from the pixel (eq. finalpixelflux).
 *   merge: segment i+1 is folded into i when flagged, outermost first, with
 *          T(i, i+1) = R_i^2 / R_(i+1)^2 on L^_thin, A^_thin and Q^_thick
 *          (reading of "Q^_thin", which the paper never defines);
 *   tau_thin,i = A^_thin / (omega R_i^2), 0 for i = 0                  (eq. tauthin)
 *   omega_thick,i = min(Q^/V^ V^^(2/3) / R_i^2, omega)                  (eq. omegaThick)
 *   tau_thick,i = A^_thick / (omega_thick R_i^2), 0 for i = 0           (eq. opt thick)
 *   eps_i = exp(-sum_(j<i) tau_thin,j) prod_(j<i) (1 - f_j + f_j e^(-tau_thick,j))
 *   F*_thin = (1 - e^-tau)/tau L^/(4 pi R_i^2), the factor = 1 for tau < 1e-4
 *   F*_thick = omega_thick L^_thick / V^_thick
 *   F*_i = (F*_thin A^_thin + F*_thick f A^_thick) / (A^_thin + f A^_thick),
 *          reading: F*_thin + F*_thick when the weight is zero (eq. fcombined)
 */
double or_ray_integrate(int nbins, int npix, double* Lth, double* Ath, double* Lk, double* Ak,
                        double* Vk, double* Qk, const double* R, uint64_t flag) {
    double omega = 4.0 * OR_PI / (double)npix;
    for (int i = nbins - 2; i >= 0; --i) {
        if (!((flag >> i) & 1ull)) continue;
        double T = (R[i] * R[i]) / (R[i + 1] * R[i + 1]);
        Lth[i] += T * Lth[i + 1];
        Ath[i] += T * Ath[i + 1];
        Qk[i] += T * Qk[i + 1];
        Lk[i] += Lk[i + 1];
        Ak[i] += Ak[i + 1];
        Vk[i] += Vk[i + 1];
        Lth[i + 1] = Ath[i + 1] = Qk[i + 1] = Lk[i + 1] = Ak[i + 1] = Vk[i + 1] = 0.0;
    }
    double tau_cum = 0.0, eps_k = 1.0, F = 0.0;
    for (int i = 0; i < nbins; ++i) {
        double R2 = R[i] * R[i];
        double tth = (i == 0) ? 0.0 : Ath[i] / (omega * R2);
        double wk = 0.0;
        if (Vk[i] > 0.0) {
            double cb = cbrt(Vk[i]);
            wk = (Qk[i] / Vk[i]) * (cb * cb) / R2;
            if (wk > omega) wk = omega;
        }
        double f = wk / omega;
        double tk = (i == 0 || wk == 0.0) ? 0.0 : Ak[i] / (wk * R2);
        double g = tth < 1e-4 ? 1.0 : -expm1(-tth) / tth;
        double Fthin = g * Lth[i] / (4.0 * OR_PI * R2);
        double Fthick = Vk[i] > 0.0 ? wk * Lk[i] / Vk[i] : 0.0;
        double den = Ath[i] + f * Ak[i];
        double Fs = den > 0.0 ? (Fthin * Ath[i] + Fthick * f * Ak[i]) / den : Fthin + Fthick;
        F += exp(-tau_cum) * eps_k * Fs;
        tau_cum += tth;
        eps_k *= (1.0 - f) + f * exp(-tk);
    }
    return F;
}

/*
 * Several HEALPix orientations (Sec. 7.6: with one orientation for every target the ray
 * pattern shows in the radiation field; turning the ray set from target to target spreads
 * it, at the price of one angular-kernel table per orientation).
 * k orientations with rotations rot[k][9] (row-major; orthonormal with determinant +1,
 * checked to 1e-9); orient[nleaves] (caller leaf order, may be NULL: leaf mod k) picks
 * each target's orientation. Ray h of orientation o points along R_o n_h. k = 0 goes back
 * to the single unturned grid. Returns 0, or -1 for a bad argument (nothing changed).
 */
int or_set_orientations(or_tree* t, int k, const double* rot, const uint8_t* orient) {
    if (k < 0 || k > 255 || (k > 0 && !rot)) return -1;
    for (int o = 0; o < k; ++o) {
        const double* R = rot + 9 * o;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double d = R[3 * a] * R[3 * b] + R[3 * a + 1] * R[3 * b + 1] + R[3 * a + 2] * R[3 * b + 2];
                if (fabs(d - (a == b ? 1.0 : 0.0)) > 1e-9) return -1;
            }
        double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                     R[2] * (R[3] * R[7] - R[4] * R[6]);
        if (det < 0.0) return -1;
    }
    if (orient)
        for (int64_t i = 0; i < t->nleaves; ++i)
            if ((int)orient[i] >= k) return -1;
    or_orient_free(t);
    if (k == 0) return 0;
    t->rot = (double*)malloc(sizeof(double) * 9 * (size_t)k);
    memcpy(t->rot, rot, sizeof(double) * 9 * (size_t)k);
    t->orient = (uint8_t*)malloc((size_t)t->nleaves);
    for (int64_t i = 0; i < t->nleaves; ++i) t->orient[i] = orient ? orient[i] : (uint8_t)(i % k);
    t->oalpha = (or_alpha_table*)calloc((size_t)k, sizeof(or_alpha_table));
    for (int o = 0; o < k; ++o) {
        t->oalpha[o].npix = t->p.npix;
        t->oalpha[o].s = t->p.alpha_s;
        t->oalpha[o].keys = (uint64_t*)calloc(OR_HCAP, sizeof(uint64_t));
        t->oalpha[o].lists = (int**)calloc(OR_HCAP, sizeof(int*));
        t->oalpha[o].rot = t->rot + 9 * o;
    }
    t->n_orient = k;
    return 0;
}

/* Angular-kernel table of a target leaf's orientation. */
static or_alpha_table* or_target_alpha(or_tree* t, int64_t leaf) {
    return t->n_orient > 0 ? &t->oalpha[t->orient[leaf]] : &t->alpha;
}

/*
 * Per-target evaluation: walk, mapping, integration and finalization.
 * Opening criterion (Sec. 4 intro): a node is opened when it appears larger than
 * theta_lim. Reading: open iff E^2 >= theta^2 d^2 (E edge, d distance from the
 * target centre to the node's geometric centre), and always open a node that
 * contains the target; leaves are always accepted.
 * Finalization (Sec. 4.4): F = sum_h -F^h n^h, J = (1/4 pi) sum_h F^h + J_src.
 * With several orientations, target leaf l uses the rays of orientation o = orient[l]:
 * its angular kernel and the directions R_o n^h.
 * targets: caller leaf indices; J[n], F[3n].
 */
int or_evaluate(or_tree* t, int64_t ntargets, const int64_t* targets, double* J, double* F,
                int nthreads) {
    const or_params* p = &t->p;
    int np = p->npix, nb = p->nbins;
    int nside = or_nside(np);
    int no = t->n_orient > 0 ? t->n_orient : 1;
    double* nhat = (double*)malloc(sizeof(double) * 3 * np * (size_t)no);
    for (int h = 0; h < np; ++h) {
        double v[3];
        or_pix2vec(nside, h, v);
        for (int o = 0; o < no; ++o) { /* orientation o: R_o n^h */
            for (int a = 0; a < 3; ++a) {
                double w = v[a];
                if (t->n_orient > 0) {
                    const double* R = t->rot + 9 * o + 3 * a;
                    w = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
                }
                nhat[3 * ((size_t)o * np + h) + a] = w;
            }
        }
    }
    double th2 = p->theta * p->theta;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        or_rays ry;
        ry.npix = np;
        ry.nbins = nb;
        size_t cells = (size_t)np * nb;
        double* buf = (double*)malloc(sizeof(double) * 6 * cells);
        ry.Lth = buf;
        ry.Ath = buf + cells;
        ry.Lk = buf + 2 * cells;
        ry.Ak = buf + 3 * cells;
        ry.Vk = buf + 4 * cells;
        ry.Qk = buf + 5 * cells;
        ry.flag = (uint64_t*)malloc(sizeof(uint64_t) * np);
        int* stack = (int*)malloc(sizeof(int) * 8 * 64 * 4);
        double R[65], Rcm[65];
        double Lr[64], Ar[64], Lkr[64], Akr[64], Vkr[64], Qkr[64];
        int myerr = 0;
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < ntargets; ++q) {
            int64_t leaf = targets[q];
            const or_node* tn = &t->nodes[t->leaf_node[leaf]];
            or_alpha_table* at = or_target_alpha(t, leaf);
            const double* nh = nhat + 3 * (size_t)np * (t->n_orient > 0 ? t->orient[leaf] : 0);
            memset(buf, 0, sizeof(double) * 6 * cells);
            memset(ry.flag, 0, sizeof(uint64_t) * np);
            or_radii(nb, t->lmax, p->periodic, p->bin_spacing, tn->E, R);
            for (int i = 0; i <= nb; ++i) Rcm[i] = R[i] * t->u;
            int sp = 0;
            stack[sp++] = 0;
            while (sp > 0) {
                int id = stack[--sp];
                const or_node* nd = &t->nodes[id];
                int64_t o[3];
                int64_t d2 = 0;
                int inside = 1;
                int ties = or_nearest(t, nd, tn, o);
                for (int a = 0; a < 3; ++a) {
                    d2 += o[a] * o[a];
                    int64_t ao = o[a] < 0 ? -o[a] : o[a];
                    if (2 * ao >= nd->E) inside = 0;
                }
                int open = 0;
                if (nd->leaf < 0) {
                    if (inside) open = 1;
                    else if ((double)(nd->E * nd->E) >= th2 * (double)d2) open = 1;
                }
                if (open) {
                    for (int k = 7; k >= 0; --k) stack[sp++] = nd->child[k];
                } else if (!ties) {
                    or_map_node(t, at, nd, o, d2, R, &ry, 1.0);
                } else { /* every closest copy, 1/2 per tied axis */
                    int nt = ((ties & 1) != 0) + ((ties & 2) != 0) + ((ties & 4) != 0);
                    double w = 1.0 / (double)(1 << nt);
                    int64_t half = (int64_t)1 << t->lmax;
                    for (int m = 0; m < 8; ++m) {
                        if (m & ~ties) continue;
                        int64_t oi[3];
                        for (int a = 0; a < 3; ++a)
                            oi[a] = ((ties >> a) & 1) ? (((m >> a) & 1) ? half : -half) : o[a];
                        or_map_node(t, at, nd, oi, d2, R, &ry, w);
                    }
                }
            }
            /* integrate every ray in CGS */
            double Jsum = 0.0, Fx = 0.0, Fy = 0.0, Fz = 0.0;
            for (int h = 0; h < np; ++h) {
                for (int i = 0; i < nb; ++i) {
                    size_t c = (size_t)i * np + h;
                    Lr[i] = ry.Lth[c];
                    Ar[i] = ry.Ath[c];
                    Lkr[i] = ry.Lk[c];
                    Akr[i] = ry.Ak[c];
                    Vkr[i] = ry.Vk[c];
                    Qkr[i] = ry.Qk[c];
                }
                double Fh = or_ray_integrate(nb, np, Lr, Ar, Lkr, Akr, Vkr, Qkr, Rcm, ry.flag[h]);
                Jsum += Fh;
                Fx -= Fh * nh[3 * h];
                Fy -= Fh * nh[3 * h + 1];
                Fz -= Fh * nh[3 * h + 2];
            }
            J[q] = Jsum / (4.0 * OR_PI) + t->Jsrc[leaf];
            F[3 * q] = Fx;
            F[3 * q + 1] = Fy;
            F[3 * q + 2] = Fz;
        }
        if (myerr) {
#pragma omp atomic write
            err = myerr;
        }
        free(buf);
        free(ry.flag);
        free(stack);
    }
    free(nhat);
    return err;
}

/*
 * Radiation energy density and pressure terms (Sec. 4.5), per leaf:
 *   u = 4 pi J / c
 *   P_dot = (F / c) kappa rho (1 - e^-tau)/tau dV, the tau factor = 1 for tau < 1e-4
 *   a_RP = P_dot / (rho dV);  force = P_dot;  P_src from the build (eq. psrc).
 * leaves: caller leaf index per row of J/F.
 */
int or_radpressure(const or_tree* t, int64_t n, const int64_t* leaves, const double* J,
                   const double* F, double* u, double* a_rp, double* force, double* p_src) {
    for (int64_t q = 0; q < n; ++q) {
        int64_t k = leaves[q];
        double dx = ldexp(t->box, -t->leaf_level[k]);
        double dV = (dx * dx) * dx;
        double tau = t->tau[k];
        double g = tau < 1e-4 ? 1.0 : -expm1(-tau) / tau;
        double kr = t->kap[k] * t->rho[k];
        u[q] = 4.0 * OR_PI * J[q] / OR_C;
        for (int a = 0; a < 3; ++a) {
            double pd = (F[3 * q + a] / OR_C) * kr * g * dV;
            force[3 * q + a] = pd;
            a_rp[3 * q + a] = (F[3 * q + a] / OR_C) * t->kap[k] * g;
        }
        p_src[q] = t->Psrc[k];
    }
    return 0;
}

/*
 * Radiation pressure of the ionising (UV) radiation on dust, neutral and ionised hydrogen
 * (Sec. 4.5, App. C), per leaf, from a given ionising photon flux N_ph (photons/s/cm^2) in
 * the unit direction u_ph and the ionised fraction x of hydrogen:
 *   P_dust = sigma_d n   (E/c) N_ph u dV,  sigma_d = 1.5e-21 cm^2 per H nucleus (Sec. 4.5)
 *   P_H    = sigma_H n_H (E/c) N_ph u dV,  n_H = (1 - x) n neutral hydrogen
 *   P_H+   = alpha_B n_p^2 (E/c) u dV,     n_p = x n protons (App. C writes n^2 for an
 *                                          ionised region)
 * with n = X rho / m_H, E = 18 eV (the mean ionising photon energy of the appendix on
 * HII-region interiors), alpha_B = 2.5e-13 cm^3/s (the Stroemgren radius of the HII-region
 * test, eq. stroemgren). The paper
 * gives no sigma_H; reading: 6.3e-18 cm^2, the hydrogen photoionisation cross-section at
 * the Lyman edge. a_uv = (P_dust + P_H + P_H+) / (rho dV); force = the sum.
 * x may be NULL (fully ionised).
 */
#define OR_SIGMA_D 1.5e-21
#define OR_SIGMA_H 6.3e-18
#define OR_ALPHA_B 2.5e-13
#define OR_EPH (18.0 * 1.602176634e-12)
int or_uv_radpressure(const or_tree* t, int64_t n, const int64_t* leaves, const double* nph,
                      const double* uph, const double* x_ion, double* a_uv, double* force) {
    for (int64_t q = 0; q < n; ++q) {
        int64_t k = leaves[q];
        double dx = ldexp(t->box, -t->leaf_level[k]);
        double dV = (dx * dx) * dx;
        double rho = t->rho[k];
        double nh = OR_XH * rho / OR_MH;
        double x = x_ion ? x_ion[q] : 1.0;
        double n0 = (1.0 - x) * nh, np = x * nh;
        double rate = OR_SIGMA_D * nh * nph[q] + OR_SIGMA_H * n0 * nph[q] + OR_ALPHA_B * np * np;
        for (int a = 0; a < 3; ++a) {
            double pd = (OR_EPH / OR_C) * rate * uph[3 * q + a] * dV;
            force[3 * q + a] = pd;
            a_uv[3 * q + a] = pd / (rho * dV);
        }
    }
    return 0;
}

/* ------------------------------------------------------ dust temperature
 * Equilibrium dust temperature (Sec. 4.6, App. D): G(T_d) = 0 with
 *   G = Gamma_dust-gas + Gamma_extra + rho kappa(T_d) (4 pi J - 4 sigma T_d^4)
 * (Gamma_BB-heat - Lambda_BB-cool with the gas-mass opacity; the dust-to-gas
 * ratio is kept in the gas-dust coupling only). Gamma_ISRF = 0 as in the paper.
 * Gamma_dust-gas uses the published Hollenbach & McKee (1989) coefficient,
 *   3.8e-33 sqrt(T) (T - T_d) (1 - 0.8 e^(-75/T)) n_H^2 (xi / 0.01) erg/s/cm^3,
 * n_H = X rho / m_H (the paper gives only the functional form).
 * Solver (the paper names none): if G(2.7 K) <= 0 the floor 2.7 K is returned;
 * otherwise hi starts at max(T_gas, T_J, 2.7) and doubles while G(hi) > 0, then
 * 60 bisections in ln T on [2.7, hi]; the result is the geometric midpoint.
 */
static double or_G(const or_params* p, double T, double rho, double Tg, double J, double H,
                   const float* kin, int64_t k) {
    double kap = or_kappa(p, T, kin, k);
    double nH = OR_XH * rho / OR_MH;
    double gd = 3.8e-33 * sqrt(Tg) * (Tg - T) * (1.0 - 0.8 * exp(-75.0 / Tg)) * (nH * nH) *
                (p->dust_to_gas / 0.01);
    double T4 = (T * T) * (T * T);
    return gd + H + rho * kap * (4.0 * OR_PI * J - 4.0 * OR_SIGMA * T4);
}

double or_td_solve(const or_params* p, double rho, double Tg, double J, double H, const float* kin,
                   int64_t k) {
    if (or_G(p, OR_TFLOOR, rho, Tg, J, H, kin, k) <= 0.0) return OR_TFLOOR;
    double TJ = sqrt(sqrt(OR_PI * (J > 0 ? J : 0.0) / OR_SIGMA));
    double hi = Tg;
    if (TJ > hi) hi = TJ;
    if (OR_TFLOOR > hi) hi = OR_TFLOOR;
    for (int it = 0; it < 64 && or_G(p, hi, rho, Tg, J, H, kin, k) > 0.0; ++it) hi *= 2.0;
    double lo = OR_TFLOOR;
    for (int it = 0; it < 60; ++it) {
        double mid = sqrt(lo * hi);
        if (or_G(p, mid, rho, Tg, J, H, kin, k) > 0.0) lo = mid;
        else hi = mid;
    }
    return sqrt(lo * hi);
}

int or_dust_temperature(const or_params* p, int64_t n, const float* rho, const float* Tgas,
                        const float* heat, const double* J, const float* kappa_in, double* Td) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k)
        Td[k] = or_td_solve(p, (double)rho[k], (double)Tgas[k], J[k], heat ? (double)heat[k] : 0.0,
                            kappa_in, k);
    return 0;
}

/* ----------------------------------------------------------- tree access */

int64_t or_tree_nnodes(const or_tree* t) { return t->nnodes; }

/* Export the canonical node list: per node level, leaf id, first child id (-1),
 * centre (3), and doubles Lt, At, Vt, LVk, Ak, Vk, m, xi, col(3) (11 per node). */
void or_tree_export(const or_tree* t, int32_t* level, int32_t* leaf, int32_t* child0,
                    int64_t* centre, double* vals) {
    for (int64_t i = 0; i < t->nnodes; ++i) {
        const or_node* nd = &t->nodes[i];
        level[i] = nd->level;
        leaf[i] = nd->leaf;
        child0[i] = nd->leaf >= 0 ? -1 : nd->child[0];
        for (int a = 0; a < 3; ++a) centre[3 * i + a] = nd->c[a];
        double* v = vals + 11 * i;
        v[0] = nd->Lt;
        v[1] = nd->At;
        v[2] = nd->Vt;
        v[3] = nd->LVk;
        v[4] = nd->Ak;
        v[5] = nd->Vk;
        v[6] = nd->m;
        v[7] = nd->xi;
        v[8] = nd->col[0];
        v[9] = nd->col[1];
        v[10] = nd->col[2];
    }
}

/* Per-leaf build outputs: kappa, tau_b, J_src, P_src, thick flag. */
void or_leaf_export(const or_tree* t, double* kap, double* tau, double* jsrc, double* psrc,
                    int32_t* thick) {
    for (int64_t k = 0; k < t->nleaves; ++k) {
        kap[k] = t->kap[k];
        tau[k] = t->tau[k];
        jsrc[k] = t->Jsrc[k];
        psrc[k] = t->Psrc[k];
        thick[k] = t->nodes[t->leaf_node[k]].thick;
    }
}

/* Accepted-node list of one target (node ids in walk order), for structure parity.
 * Returns the count; writes at most cap ids. */
int64_t or_accepted(const or_tree* t, int64_t leaf, int32_t* ids, int64_t cap) {
    const or_node* tn = &t->nodes[t->leaf_node[leaf]];
    double th2 = t->p.theta * t->p.theta;
    int stack[8 * 64 * 4];
    int sp = 0;
    int64_t n = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        int id = stack[--sp];
        const or_node* nd = &t->nodes[id];
        int64_t d2 = 0, o[3];
        int inside = 1;
        or_nearest(t, nd, tn, o);
        for (int a = 0; a < 3; ++a) {
            d2 += o[a] * o[a];
            if (2 * (o[a] < 0 ? -o[a] : o[a]) >= nd->E) inside = 0;
        }
        int open = nd->leaf < 0 && (inside || (double)(nd->E * nd->E) >= th2 * (double)d2);
        if (open) {
            for (int k = 7; k >= 0; --k) stack[sp++] = nd->child[k];
        } else {
            if (n < cap) ids[n] = id;
            ++n;
        }
    }
    return n;
}

/* Angular key of an accepted node at offset o: at its geometric centre (or_key), or with
 * COL mapping, for a node whose COL is off centre, the odd grid point of its COL position
 * in FP64 (as in or_map_node). */
static void or_node_key(const or_tree* t, const or_node* nd, const int64_t* o, int64_t* K) {
    if (t->p.col_mapping) {
        double pc[3];
        int shifted = 0;
        for (int a = 0; a < 3; ++a) {
            double c = nd->col[a] - (double)nd->c[a];
            if (c != 0.0) shifted = 1;
            pc[a] = (double)o[a] + c;
        }
        if (shifted) {
            for (int a = 0; a < 3; ++a) K[a] = 2 * (int64_t)floor(4.0 * pc[a] / (double)nd->E) + 1;
            return;
        }
    }
    or_key(o, nd->E, K);
}

/* Walk statistics of one target: nodes visited (tested against the opening
 * criterion), nodes accepted (own cell included) and angular-kernel entries read by
 * the accepted nodes other than the own cell. out[3]. */
void or_walk_stats(or_tree* t, int64_t leaf, int64_t* out) {
    const or_node* tn = &t->nodes[t->leaf_node[leaf]];
    double th2 = t->p.theta * t->p.theta;
    int stack[8 * 64 * 4];
    int sp = 0;
    int64_t visits = 0, acc = 0, ent = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        int id = stack[--sp];
        const or_node* nd = &t->nodes[id];
        ++visits;
        int64_t o[3], d2 = 0;
        int inside = 1;
        int ties = or_nearest(t, nd, tn, o);
        for (int a = 0; a < 3; ++a) {
            d2 += o[a] * o[a];
            if (2 * (o[a] < 0 ? -o[a] : o[a]) >= nd->E) inside = 0;
        }
        int open = nd->leaf < 0 && (inside || (double)(nd->E * nd->E) >= th2 * (double)d2);
        if (open) {
            for (int k = 7; k >= 0; --k) stack[sp++] = nd->child[k];
        } else {
            ++acc;
            if (d2 != 0) {
                int64_t half = (int64_t)1 << t->lmax;
                for (int m = 0; m < 8; ++m) { /* entries of every closest copy */
                    if (m & ~ties) continue;
                    int64_t oi[3], K[3];
                    for (int a = 0; a < 3; ++a)
                        oi[a] = ((ties >> a) & 1) ? (((m >> a) & 1) ? half : -half) : o[a];
                    int owned = 0;
                    or_node_key(t, nd, oi, K);
                    const int* l = or_alpha_get(or_target_alpha(t, leaf), K, &owned);
                    int n = 0;
                    while (l[2 * n] >= 0) ++n;
                    ent += n;
                    if (owned) free((void*)l);
                }
            }
        }
    }
    out[0] = visits;
    out[1] = acc;
    out[2] = ent;
}

/* Evaluation radii R_i (half-units) for a target leaf. */
void or_target_radii(const or_tree* t, int64_t leaf, double* R) {
    or_radii(t->p.nbins, t->lmax, t->p.periodic, t->p.bin_spacing, t->nodes[t->leaf_node[leaf]].E, R);
}

/* alpha key for an offset o and node edge E. */
void or_alpha_key(const int64_t* o, int64_t E, int64_t* K) { or_key(o, E, K); }

double or_unit_cm(const or_tree* t) { return t->u; }

/*
 * Long-characteristic brute force on a uniform n^3 grid (independent of the tree):
 *   J = sum_k L_k e^(-tau_k) / (16 pi^2 r_k^2),  F = sum_k L_k e^(-tau_k) (-r_k^) / (4 pi r_k^2)
 * where L_k = L_thin of cell k (+S), r_k the centre distance, and tau_k the exact
 * optical depth along the straight line between the centres through the cells'
 * rho kappa (3-D DDA); the target's own cell is excluded. Thin media only.
 */
int or_brute_lc(int n, double box, const double* Lcell, const double* ak /* rho kappa */,
                int64_t nt, const int64_t* targets, int with_ext, double* J, double* F) {
    double dx = box / n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < nt; ++q) {
        int64_t tk = targets[q];
        int ti = (int)(tk % n), tj = (int)((tk / n) % n), tl = (int)(tk / ((int64_t)n * n));
        double P0[3] = {(ti + 0.5) * dx, (tj + 0.5) * dx, (tl + 0.5) * dx};
        double Js = 0, Fx = 0, Fy = 0, Fz = 0;
        for (int64_t k = 0; k < (int64_t)n * n * n; ++k) {
            if (k == tk || Lcell[k] == 0.0) continue;
            int ci = (int)(k % n), cj = (int)((k / n) % n), cl = (int)(k / ((int64_t)n * n));
            double P1[3] = {(ci + 0.5) * dx, (cj + 0.5) * dx, (cl + 0.5) * dx};
            double dvec[3] = {P1[0] - P0[0], P1[1] - P0[1], P1[2] - P0[2]};
            double r = sqrt(dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2]);
            double tau = 0.0;
            if (with_ext) {
                /* DDA from P0 to P1 */
                int cell[3] = {ti, tj, tl};
                int step[3];
                double tmax[3], tdel[3];
                for (int a = 0; a < 3; ++a) {
                    if (dvec[a] > 0) {
                        step[a] = 1;
                        tmax[a] = ((cell[a] + 1) * dx - P0[a]) / dvec[a];
                        tdel[a] = dx / dvec[a];
                    } else if (dvec[a] < 0) {
                        step[a] = -1;
                        tmax[a] = (cell[a] * dx - P0[a]) / dvec[a];
                        tdel[a] = -dx / dvec[a];
                    } else {
                        step[a] = 0;
                        tmax[a] = 1e300;
                        tdel[a] = 1e300;
                    }
                }
                double tcur = 0.0;
                for (;;) {
                    int a = 0;
                    if (tmax[1] < tmax[a]) a = 1;
                    if (tmax[2] < tmax[a]) a = 2;
                    double tn = tmax[a] < 1.0 ? tmax[a] : 1.0;
                    int64_t idx = cell[0] + (int64_t)n * (cell[1] + (int64_t)n * cell[2]);
                    tau += ak[idx] * (tn - tcur) * r;
                    if (tn >= 1.0) break;
                    tcur = tn;
                    cell[a] += step[a];
                    tmax[a] += tdel[a];
                    if (cell[a] < 0 || cell[a] >= n) break;
                }
            }
            double w = Lcell[k] * exp(-tau) / (4.0 * OR_PI * r * r);
            Js += w / (4.0 * OR_PI);
            Fx -= w * dvec[0] / r;
            Fy -= w * dvec[1] / r;
            Fz -= w * dvec[2] / r;
        }
        J[q] = Js;
        F[3 * q] = Fx;
        F[3 * q + 1] = Fy;
        F[3 * q + 2] = Fz;
    }
    return 0;
}
