// Tree build on the GPU (Sec. 4.1 and App. A of Klepitko et al. 2023):
//   1. per leaf: Morton key of its lower corner at the finest level, prefixed by its level;
//   2. stable LSD radix sort of the keys with the leaf permutation;
//   3. level-synchronous node construction, deepest level first: the h-nodes of level l
//      are every 8th entry of level l+1 (a complete octree), merged with the leaves of
//      level l by key;
//   4. b-node quantities in FP64 (eqs. lthinbnode, athinbnode, lthickbnode, S, J_src, P_src);
//   5. upward sums in FP64 in Morton child order and the centre of luminosity (eq. COL);
//   6. FP32 walk records in internal units (luminosity / L_scale, lengths in half-cells).
// This file is compiled with -fmad=false: every FP64 sum and product is rounded as
// written, so node moments reproduce a plain sequential FP64 evaluation exactly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace tr {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortTile = 4096;  // keys per block and pass

__host__ __device__ inline uint64_t morton3(uint64_t x, uint64_t y, uint64_t z, int bits) {
    uint64_t k = 0;
    for (int b = 0; b < bits; ++b)
        k |= (((x >> b) & 1ull) << (3 * b)) | (((y >> b) & 1ull) << (3 * b + 1)) |
             (((z >> b) & 1ull) << (3 * b + 2));
    return k;
}

// Level and integer coordinates (at that level) of caller leaf k.
struct LeafGrid {
    int n;               // uniform cells per axis, 0 for AMR
    int lmax;
    const int4* blocks;  // AMR: (bi, bj, bk, level)
};

__device__ inline void leaf_coords(const LeafGrid& g, int64_t k, int* lvl, int64_t* ijk) {
    if (g.n > 0) {
        ijk[0] = k % g.n;
        ijk[1] = (k / g.n) % g.n;
        ijk[2] = k / ((int64_t)g.n * g.n);
        *lvl = g.lmax;
    } else {
        const int4 b = g.blocks[k >> 9];
        const int c = (int)(k & 511);
        ijk[0] = 8 * (int64_t)b.x + (c & 7);
        ijk[1] = 8 * (int64_t)b.y + ((c >> 3) & 7);
        ijk[2] = 8 * (int64_t)b.z + (c >> 6);
        *lvl = b.w;
    }
}

__global__ void k_leaf_keys(LeafGrid g, int64_t n, uint64_t* keys, int32_t* vals) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int l;
    int64_t c[3];
    leaf_coords(g, k, &l, c);
    const int sh = g.lmax - l;
    keys[k] = ((uint64_t)l << (3 * g.lmax)) |
              morton3((uint64_t)c[0] << sh, (uint64_t)c[1] << sh, (uint64_t)c[2] << sh, g.lmax);
    vals[k] = (int32_t)k;
}

// ---- stable LSD radix sort, 8-bit digits
__global__ void k_rs_hist(const uint64_t* keys, int64_t n, int shift, uint32_t* hist, int nb) {
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int j = threadIdx.x; j < kSortTile; j += blockDim.x) {
        const int64_t i = base + j;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * nb + blockIdx.x] = h[d];
}

// Block-wide exclusive scan of one value per thread (256 threads); returns the total.
__device__ inline uint32_t block_scan_256(uint32_t v, uint32_t* sh, uint32_t* out_excl) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        const uint32_t x = t >= off ? sh[t - off] : 0u;
        __syncthreads();
        sh[t] += x;
        __syncthreads();
    }
    *out_excl = sh[t] - v;
    const uint32_t total = sh[255];
    __syncthreads();
    return total;
}

// Row d of the histogram ([256 digits][nb blocks]): exclusive scan in place, row total
// to rowsum[d]. One block of 256 threads per digit.
__global__ void __launch_bounds__(256) k_rs_scan_rows(uint32_t* hist, int nb, uint32_t* rowsum) {
    __shared__ uint32_t sh[256];
    uint32_t* row = hist + (int64_t)blockIdx.x * nb;
    const int per = (nb + 255) / 256;
    const int lo = threadIdx.x * per, hi = min(nb, lo + per);
    uint32_t s = 0;
    for (int i = lo; i < hi; ++i) s += row[i];
    uint32_t ex;
    const uint32_t total = block_scan_256(s, sh, &ex);
    for (int i = lo; i < hi; ++i) {
        const uint32_t v = row[i];
        row[i] = ex;
        ex += v;
    }
    if (threadIdx.x == 0) rowsum[blockIdx.x] = total;
}

// exclusive scan of the 256 digit totals in place (one block of 256 threads)
__global__ void __launch_bounds__(256) k_rs_scan_digits(uint32_t* rowsum) {
    __shared__ uint32_t sh[256];
    uint32_t ex;
    block_scan_256(rowsum[threadIdx.x], sh, &ex);
    rowsum[threadIdx.x] = ex;
}

__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(const uint64_t* kin, const int32_t* vin,
                                                             uint64_t* kout, int32_t* vout, int64_t n,
                                                             int shift, const uint32_t* hist, int nb,
                                                             const uint32_t* digit_base) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wc[kSortThreads / 32][257];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int d = t; d < 256; d += blockDim.x) base[d] = digit_base[d] + hist[(int64_t)d * nb + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int c = 0; c < kSortTile / kSortThreads; ++c) {
        for (int i = t; i < (kSortThreads / 32) * 257; i += blockDim.x) (&wc[0][0])[i] = 0;
        __syncthreads();
        const int64_t i = (int64_t)blockIdx.x * kSortTile + (int64_t)c * kSortThreads + t;
        const bool valid = i < n;
        uint64_t key = 0;
        int32_t val = 0;
        int d = 256;
        if (valid) {
            key = kin[i];
            val = vin[i];
            d = (int)((key >> shift) & 255u);
        }
        const unsigned same = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(same & lt_mask);
        if (rank == 0) wc[warp][d] = __popc(same);
        __syncthreads();
        if (valid) {
            uint32_t pre = 0;
            for (int w = 0; w < warp; ++w) pre += wc[w][d];
            const uint32_t pos = base[d] + pre + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        for (int dd = t; dd < 256; dd += blockDim.x) {
            uint32_t tot = 0;
            for (int w = 0; w < kSortThreads / 32; ++w) tot += wc[w][dd];
            base[dd] += tot;
        }
        __syncthreads();
    }
}

__global__ void k_inverse(const int32_t* perm, int64_t n, int32_t* inv) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < n) inv[perm[s]] = (int32_t)s;
}

__global__ void k_level_bounds(const uint64_t* keys, int64_t n, int lmax, int* lo, int* hi) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int l = (int)(keys[s] >> (3 * lmax));
    if (s == 0 || (int)(keys[s - 1] >> (3 * lmax)) != l) lo[l] = (int)s;
    if (s == n - 1 || (int)(keys[s + 1] >> (3 * lmax)) != l) hi[l] = (int)s + 1;
}

__device__ inline uint64_t leaf_prefix(const uint64_t* keys, int64_t s, int lmax, int l) {
    const uint64_t m = keys[s] & ((1ull << (3 * lmax)) - 1ull);
    return m >> (3 * (lmax - l));
}

// child node of an internal node at level l starts at off1 + 8 j
__device__ inline uint64_t internal_prefix(const uint64_t* prefix, int64_t off1, int64_t j) {
    return prefix[off1 + 8 * j] >> 3;
}

struct LevelArgs {
    const uint64_t* keys;
    uint64_t* prefix;
    int4* geo;
    int32_t* leaf_node;
    int lmax, l;
    int64_t off, off1;      // first node of level l and of level l+1
    int64_t nint, nleaf;    // internal nodes and leaves at level l
    int64_t leaf_lo;        // first sorted leaf of level l
};

__device__ inline void write_node(const LevelArgs& a, int64_t pos, uint64_t p, int32_t child) {
    const int64_t id = a.off + pos;
    a.prefix[id] = p;
    // geometric centre in half-cells of the finest level: (2 a + 1) E / 2, E = 2^(lmax-l+1)
    uint64_t x = 0, y = 0, z = 0;
    for (int b = 0; b < a.l; ++b) {
        x |= ((p >> (3 * b)) & 1ull) << b;
        y |= ((p >> (3 * b + 1)) & 1ull) << b;
        z |= ((p >> (3 * b + 2)) & 1ull) << b;
    }
    const int64_t half = (int64_t)1 << (a.lmax - a.l);
    int4 g;
    g.x = (int)((2 * (int64_t)x + 1) * half);
    g.y = (int)((2 * (int64_t)y + 1) * half);
    g.z = (int)((2 * (int64_t)z + 1) * half) | (a.l << 24);
    g.w = child;
    a.geo[id] = g;
    if (child < 0) a.leaf_node[-1 - child] = (int32_t)id;
}

__global__ void k_level_internal(LevelArgs a) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= a.nint) return;
    const uint64_t p = internal_prefix(a.prefix, a.off1, j);
    // number of leaves of this level with a smaller prefix
    int64_t lo = 0, hi = a.nleaf;
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        if (leaf_prefix(a.keys, a.leaf_lo + m, a.lmax, a.l) < p) lo = m + 1;
        else hi = m;
    }
    write_node(a, j + lo, p, (int32_t)(a.off1 + 8 * j));
}

__global__ void k_level_leaves(LevelArgs a) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= a.nleaf) return;
    const uint64_t p = leaf_prefix(a.keys, a.leaf_lo + m, a.lmax, a.l);
    int64_t lo = 0, hi = a.nint;
    while (lo < hi) {
        const int64_t mm = (lo + hi) >> 1;
        if (internal_prefix(a.prefix, a.off1, mm) < p) lo = mm + 1;
        else hi = mm;
    }
    write_node(a, m + lo, p, (int32_t)(-1 - (a.leaf_lo + m)));
}

// Structure validation before any kernel follows child links: every internal node of
// level l owns 8 children at level l+1 aligned to a multiple of 8 with prefixes
// 8p .. 8p+7, and every leaf slot points at a leaf that points back at it. Slots
// never written (invalid input) fail one of the two tests.
__global__ void k_check_nodes(const uint64_t* prefix, const int4* geo, const int32_t* leaf_node,
                              int64_t off, int64_t cnt, int64_t off1, int64_t cnt1, int64_t nleaves,
                              unsigned* err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int4 g = geo[off + i];
    if (g.w >= 0) {
        const int64_t c0 = g.w;
        if (c0 < off1 || c0 + 8 > off1 + cnt1 || ((c0 - off1) & 7) != 0) {
            atomicOr(err, kErrOctree);
            return;
        }
        const uint64_t p = prefix[off + i];
        for (int c = 0; c < 8; ++c)
            if (prefix[c0 + c] != ((p << 3) | (uint64_t)c)) atomicOr(err, kErrOctree);
    } else {
        const int64_t s = -1 - (int64_t)g.w;
        if (s >= nleaves || leaf_node[s] != off + i) atomicOr(err, kErrOctree);
    }
}

__global__ void k_check_leaves(const int32_t* leaf_node, int64_t nleaves, int64_t nn, unsigned* err) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nleaves) return;
    const int32_t v = leaf_node[s];
    if (v < 0 || v >= nn) atomicOr(err, kErrOctree);
}

struct MomArgs {
    LeafGrid g;
    const int32_t* perm;
    const int32_t* leaf_node;
    const float* rho;
    const float* Td;
    const float* kin;
    const double* star;  // [n_stars][4]: x, y, z, L
    int n_stars;
    double box;
    int model;
    double kappa0, kext;
    int emit;
    int64_t nn, nleaves;
    double* mom;         // [11][nn]
    const int4* geo;
    double* kap;
    double* tau;
    double* jsrc;
    double* psrc;
    int32_t* thick;
    float* rho_copy;
    float* kin_copy;
    const int* skip;     // fixed-point mode: return at once when *skip != 0
    unsigned* err;       // device error word: kErrInput for a negative or non-finite input
};

// b-node quantities (Sec. 4.1.1); expression order fixed (see the file header)
__global__ void k_leaf_moments(MomArgs a) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= a.nleaves || (a.skip && *a.skip)) return;
    const int64_t k = a.perm[s];
    const int64_t node = a.leaf_node[s];
    int l;
    int64_t c[3];
    leaf_coords(a.g, k, &l, c);
    const double T = (double)a.Td[k];
    const double rh = (double)a.rho[k];
    double kap;
    if (a.kin) kap = (double)a.kin[k];
    else if (a.model == 0) kap = a.kappa0;
    else {
        const double Tc = T < 150.0 ? T : 150.0;
        kap = 1.0e-3 * (Tc * Tc);
    }
    // inputs outside their domain (negative or NaN/inf) are reported, not used to index
    // anything; the results of such a build are undefined
    if (!(rh >= 0.0 && rh <= 3.4e38) || !(T >= 0.0 && T <= 3.4e38) || !(kap >= 0.0 && kap <= 3.4e38))
        atomicOr(a.err, kErrInput);
    const double dx = ldexp(a.box, -l);
    const double dV = (dx * dx) * dx;
    const double rk = rh * kap;
    const double tau = rk * dx;
    const int th = tau >= 1.0;
    const double T4 = (T * T) * (T * T);
    const double A = (rk * dV) * a.kext;
    // stars hosted by this leaf, summed in input order
    double Ls = 0.0;
    const double dxf = ldexp(a.box, -a.g.lmax);
    const int64_t fmax = ((int64_t)1 << a.g.lmax) - 1;
    const int sh = a.g.lmax - l;
    for (int q = 0; q < a.n_stars; ++q) {
        bool in = true;
        for (int ax = 0; ax < 3; ++ax) {
            const double f = floor(a.star[4 * q + ax] / dxf);
            int64_t fi = (int64_t)f;
            if (f < 0) fi = 0;
            if (f > (double)fmax) fi = fmax;
            in = in && ((fi >> sh) == c[ax]);
        }
        if (in) Ls += a.star[4 * q + 3];
    }
    const double ext = exp(-0.5 * tau);
    const double S = Ls * ext;
    a.kap[k] = kap;
    a.tau[k] = tau;
    a.jsrc[k] = ((1.0 - ext) * Ls) / (dx * dx);
    a.psrc[k] = ((1.0 - ext) * Ls) / (kLightC * (dx * dx));
    a.thick[k] = th;
    a.rho_copy[k] = a.rho[k];
    if (a.kin_copy) a.kin_copy[k] = a.kin[k];
    double Lt, At, Vt, LVk, Ak, Vk, xi;
    if (!th) {
        const double L = a.emit ? (((4.0 * kSigmaSB) * rk) * T4) * dV : 0.0;
        Lt = L + S;
        At = A;
        Vt = dV;
        LVk = Ak = Vk = 0.0;
        xi = Lt;
    } else {
        const double Lu = a.emit ? (kSigmaSB / kPi) * T4 : 0.0;
        Lt = S;
        At = 0.0;
        Vt = 0.0;
        LVk = Lu * dV;
        Ak = A;
        Vk = dV;
        xi = S + Lu * (dx * dx);
    }
    const int64_t nn = a.nn;
    const int4 g = a.geo[node];
    a.mom[0 * nn + node] = Lt;
    a.mom[1 * nn + node] = At;
    a.mom[2 * nn + node] = Vt;
    a.mom[3 * nn + node] = LVk;
    a.mom[4 * nn + node] = Ak;
    a.mom[5 * nn + node] = Vk;
    a.mom[6 * nn + node] = rh * dV;
    a.mom[7 * nn + node] = xi;
    a.mom[8 * nn + node] = (double)g.x;
    a.mom[9 * nn + node] = (double)g.y;
    a.mom[10 * nn + node] = (double)(g.z & 0xffffff);
}

// upward propagation (App. A) for the internal nodes of one level
__global__ void k_internal_moments(const int4* geo, double* mom, int64_t nn, int64_t off, int64_t cnt,
                                   const int* skip) {
    const int64_t i = off + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= off + cnt || (skip && *skip)) return;
    const int4 g = geo[i];
    if (g.w < 0) return;
    double Lt = 0.0, At = 0.0, Vt = 0.0, LVk = 0.0, Ak = 0.0, Vk = 0.0, m = 0.0;
    double Xi = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
    for (int k = 0; k < 8; ++k) {
        const int64_t ch = g.w + k;
        const double xi = mom[7 * nn + ch];
        Lt = Lt + mom[0 * nn + ch];
        At = At + mom[1 * nn + ch];
        Vt = Vt + mom[2 * nn + ch];
        LVk = LVk + mom[3 * nn + ch];
        Ak = Ak + mom[4 * nn + ch];
        Vk = Vk + mom[5 * nn + ch];
        m = m + mom[6 * nn + ch];
        Xi = Xi + xi;
        cx = cx + xi * mom[8 * nn + ch];
        cy = cy + xi * mom[9 * nn + ch];
        cz = cz + xi * mom[10 * nn + ch];
    }
    double xi_self = Lt;
    if (Vk > 0.0) {
        const double cb = cbrt(Vk);
        xi_self = Lt + (LVk / Vk) * (cb * cb);
    }
    mom[0 * nn + i] = Lt;
    mom[1 * nn + i] = At;
    mom[2 * nn + i] = Vt;
    mom[3 * nn + i] = LVk;
    mom[4 * nn + i] = Ak;
    mom[5 * nn + i] = Vk;
    mom[6 * nn + i] = m;
    mom[7 * nn + i] = xi_self;
    if (Xi > 0.0) {
        mom[8 * nn + i] = cx / Xi;
        mom[9 * nn + i] = cy / Xi;
        mom[10 * nn + i] = cz / Xi;
    } else {
        mom[8 * nn + i] = (double)g.x;
        mom[9 * nn + i] = (double)g.y;
        mom[10 * nn + i] = (double)(g.z & 0xffffff);
    }
}

// luminosity scale: a power of two at or above the largest of the root's thin luminosity
// and its thick L_ V / u, so that FP32 node records stay far from overflow
__global__ void k_scale(const double* mom, int64_t nn, double u, double* scal, const int* skip) {
    if (skip && *skip) return;
    double m = mom[0];
    const double t = mom[3 * nn] / u;
    if (t > m) m = t;
    int e = 0;
    if (m > 0.0) {
        frexp(m, &e);
        scal[0] = ldexp(1.0, e);
    } else {
        scal[0] = 1.0;
    }
}

// FP32 walk records in internal units: luminosity / L_scale, area / u^2, volume / u^3,
// thick sum L_ V / (L_scale u), COL offsets from the geometric centre in half-cells
__global__ void k_pack(const int4* geo, const double* mom, int64_t nn, double u, const double* scal,
                       float4* thin, float4* thick, const int* skip) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nn || (skip && *skip)) return;
    // the FP32 walk records: scaled by reciprocals (the GB300's FP64 division is slow; the
    // scaled values differ from quotients by at most an FP64 rounding before the FP32 one,
    // and 1 / L_scale is exact, L_scale being a power of two)
    const double iLs = 1.0 / scal[0];
    const double iu = 1.0 / u, iu2 = iu * iu, iu3 = iu2 * iu;
    const int4 g = geo[i];
    const double ox = mom[8 * nn + i] - (double)g.x;
    const double oy = mom[9 * nn + i] - (double)g.y;
    const double oz = mom[10 * nn + i] - (double)(g.z & 0xffffff);
    thin[i] = make_float4((float)(mom[0 * nn + i] * iLs), (float)(mom[1 * nn + i] * iu2), (float)ox, (float)oy);
    thick[i] = make_float4((float)oz, (float)((mom[3 * nn + i] * iLs) * iu), (float)(mom[4 * nn + i] * iu2),
                           (float)(mom[5 * nn + i] * iu3));
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

template <typename T>
treeray_status grow(treeray_ctx* c, T** p, int64_t* cap, int64_t need) {
    if (*p && *cap >= need) return TREERAY_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    return dev_alloc(c, (void**)p, sizeof(T) * std::max<int64_t>(need, 1));
}

}  // namespace

void free_tree(DeviceTree& t) {
    void* ptrs[] = {t.geo,  t.thin, t.thick,     t.mom,      t.prefix, t.keys,     t.perm,
                    t.inv_perm, t.leaf_node, t.kap, t.tau, t.jsrc, t.psrc, t.thickflag,
                    t.rho,  t.kin,  t.keys_alt,  t.vals_alt, t.hist, t.stars, t.blocks, t.levels};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    t = DeviceTree{};
}

treeray_status build_tree(treeray_ctx* c, const treeray_grid* gr, const float* rho, const float* Td,
                          const float* kappa, int n_stars, const double* star_pos,
                          const double* star_lum, cudaStream_t st) {
    DeviceTree& T = c->tree;
    // ---- grid validation
    int lmax = 0;
    int64_t N = 0;
    std::vector<int4> hblocks;
    if (gr->n < 0) {
        set_error("grid: n must be a power of two (uniform) or 0 (AMR blocks)");
        return TREERAY_EINVAL;
    }
    if (gr->n > 0) {
        if (gr->n_blocks != 0) {
            set_error("grid: give either n (uniform) or n_blocks (AMR), not both");
            return TREERAY_EINVAL;
        }
        int n = gr->n;
        while ((1 << lmax) < n) ++lmax;
        if ((1 << lmax) != n || lmax > 10) {
            set_error("grid: n must be a power of two <= 1024");
            return TREERAY_EINVAL;
        }
        N = (int64_t)n * n * n;
    } else {
        if (gr->n_blocks <= 0 || !gr->blocks) {
            set_error("grid: n_blocks must be positive with a host blocks array");
            return TREERAY_EINVAL;
        }
        hblocks.resize(gr->n_blocks);
        for (int b = 0; b < gr->n_blocks; ++b) {
            const int32_t* q = gr->blocks + 4 * b;
            if (q[3] < 3 || q[3] > kMaxLevel) {
                set_error("grid: AMR cell levels must lie in 3.." + std::to_string(kMaxLevel));
                return TREERAY_EINVAL;
            }
            const int64_t nb = (int64_t)1 << (q[3] - 3);
            for (int a = 0; a < 3; ++a)
                if (q[a] < 0 || q[a] >= nb) {
                    set_error("grid: AMR block coordinates outside the box");
                    return TREERAY_EINVAL;
                }
            hblocks[b] = make_int4(q[0], q[1], q[2], q[3]);
            lmax = std::max(lmax, (int)q[3]);
        }
        N = (int64_t)gr->n_blocks * 512;
    }
    if (!(gr->box > 0)) {
        set_error("grid: box must be positive");
        return TREERAY_EINVAL;
    }
    if (N > (int64_t)1 << 30) {
        set_error("grid: too many leaves");
        return TREERAY_EINVAL;
    }
    if (n_stars < 0 || n_stars > kMaxStars || (n_stars > 0 && (!star_pos || !star_lum))) {
        set_error("stars: 0..4096 with host position and luminosity arrays");
        return TREERAY_EINVAL;
    }
    for (int q = 0; q < n_stars; ++q) {
        const double x = star_pos[3 * q], y = star_pos[3 * q + 1], z = star_pos[3 * q + 2], L = star_lum[q];
        if (!(std::isfinite(x) && std::isfinite(y) && std::isfinite(z) && L >= 0.0 && std::isfinite(L))) {
            set_error("stars: positions must be finite and luminosities finite and >= 0");
            return TREERAY_EINVAL;
        }
    }
    if (!rho || !Td) {
        set_error("rho and Td are required");
        return TREERAY_EINVAL;
    }
    c->built = false;
    c->amr = gr->n == 0;
    c->lmax = lmax;
    c->box = gr->box;
    c->u = ldexp(gr->box, -(lmax + 1));
    c->nleaves = N;

    // ---- leaf buffers
    treeray_status rc;
    int64_t cl = T.cap_leaves;
#define GROW(ptr, need, capv)                                   \
    do {                                                        \
        int64_t cc_ = (capv);                                   \
        if ((rc = grow(c, &(ptr), &cc_, (need))) != TREERAY_OK) return rc; \
    } while (0)
    GROW(T.keys, N, cl);
    GROW(T.keys_alt, N, cl);
    GROW(T.perm, N, cl);
    GROW(T.vals_alt, N, cl);
    GROW(T.inv_perm, N, cl);
    GROW(T.leaf_node, N, cl);
    GROW(T.kap, N, cl);
    GROW(T.tau, N, cl);
    GROW(T.jsrc, N, cl);
    GROW(T.psrc, N, cl);
    GROW(T.thickflag, N, cl);
    GROW(T.rho, N, cl);
    GROW(T.kin, N, cl);
    T.cap_leaves = std::max(T.cap_leaves, N);

    std::vector<double> hst(4 * (size_t)std::max(n_stars, 1));
    for (int q = 0; q < n_stars; ++q) {
        hst[4 * q + 0] = star_pos[3 * q + 0];
        hst[4 * q + 1] = star_pos[3 * q + 1];
        hst[4 * q + 2] = star_pos[3 * q + 2];
        hst[4 * q + 3] = star_lum[q];
    }
    {
        int64_t cs = T.cap_stars;
        if ((rc = grow(c, &T.stars, &cs, (int64_t)hst.size())) != TREERAY_OK) return rc;
        T.cap_stars = std::max(T.cap_stars, (int64_t)hst.size());
        int64_t cv = T.levels ? 2 * (kMaxLevel + 1) : 0;
        if ((rc = grow(c, &T.levels, &cv, 2 * (kMaxLevel + 1))) != TREERAY_OK) return rc;
        if (c->amr) {
            int64_t cb = T.cap_blocks;
            if ((rc = grow(c, &T.blocks, &cb, (int64_t)hblocks.size())) != TREERAY_OK) return rc;
            T.cap_blocks = std::max(T.cap_blocks, (int64_t)hblocks.size());
        }
    }
    int4* dblocks = T.blocks;
    double* dstars = T.stars;
    int* dlev = T.levels;
    // host staging buffers must stay alive until their copies have run
    TR_CUDA(cudaMemcpyAsync(dstars, hst.data(), sizeof(double) * hst.size(), cudaMemcpyHostToDevice, st));
    if (c->amr)
        TR_CUDA(cudaMemcpyAsync(dblocks, hblocks.data(), sizeof(int4) * hblocks.size(),
                                cudaMemcpyHostToDevice, st));
    LeafGrid lg{gr->n, lmax, dblocks};

    // ---- keys and sort
    k_leaf_keys<<<nblk(N, 256), 256, 0, st>>>(lg, N, T.keys, T.perm);
    ++c->launches;
    const int nbk = nblk(N, kSortTile);
    const int64_t nh = 256 * (int64_t)nbk;
    int64_t ch = T.cap_hist;
    if ((rc = grow(c, &T.hist, &ch, nh + 256)) != TREERAY_OK) return rc;
    T.cap_hist = std::max(T.cap_hist, nh + 256);
    uint32_t* digit_base = T.hist + nh;
    const int bits = 3 * lmax + 5;
    uint64_t* ka = T.keys;
    int32_t* va = T.perm;
    uint64_t* kb = T.keys_alt;
    int32_t* vb = T.vals_alt;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8, ++passes) {
        k_rs_hist<<<nbk, kSortThreads, 0, st>>>(ka, N, shift, T.hist, nbk);
        ++c->launches;
        k_rs_scan_rows<<<256, 256, 0, st>>>(T.hist, nbk, digit_base);
        ++c->launches;
        k_rs_scan_digits<<<1, 256, 0, st>>>(digit_base);
        ++c->launches;
        k_rs_scatter<<<nbk, kSortThreads, 0, st>>>(ka, va, kb, vb, N, shift, T.hist, nbk, digit_base);
        ++c->launches;
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {  // result must end in T.keys / T.perm
        TR_CUDA(cudaMemcpyAsync(T.keys, ka, sizeof(uint64_t) * N, cudaMemcpyDeviceToDevice, st));
        TR_CUDA(cudaMemcpyAsync(T.perm, va, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
    }
    k_inverse<<<nblk(N, 256), 256, 0, st>>>(T.perm, N, T.inv_perm);
    ++c->launches;

    // ---- leaves per level (one host round trip sizes the tree)
    std::vector<int> hl(2 * (kMaxLevel + 1), 0);
    TR_CUDA(cudaMemsetAsync(dlev, 0, sizeof(int) * 2 * (kMaxLevel + 1), st));
    k_level_bounds<<<nblk(N, 256), 256, 0, st>>>(T.keys, N, lmax, dlev, dlev + kMaxLevel + 1);
    ++c->launches;
    TR_CUDA(cudaMemcpyAsync(hl.data(), dlev, sizeof(int) * hl.size(), cudaMemcpyDeviceToHost, st));
    TR_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> nleaf(lmax + 1, 0), llo(lmax + 1, 0), nint(lmax + 1, 0), nent(lmax + 1, 0);
    for (int l = 0; l <= lmax; ++l) {
        llo[l] = hl[l];
        nleaf[l] = std::max(0, hl[kMaxLevel + 1 + l] - hl[l]);
    }
    for (int l = lmax; l >= 0; --l) {
        if (l == lmax) nint[l] = 0;
        else {
            if (nent[l + 1] % 8 != 0) {
                set_error("grid: leaves do not form a complete octree");
                return TREERAY_EINVAL;
            }
            nint[l] = nent[l + 1] / 8;
        }
        nent[l] = nint[l] + nleaf[l];
    }
    if (nent[0] != 1) {
        set_error("grid: leaves do not form a complete octree (root)");
        return TREERAY_EINVAL;
    }
    int64_t nn = 0;
    for (int l = 0; l <= lmax; ++l) {
        c->level_off[l] = (int)nn;
        c->level_cnt[l] = (int)nent[l];
        nn += nent[l];
    }
    if (nn >= ((int64_t)1 << 27)) {
        set_error("grid: more than 2^27 tree nodes");
        return TREERAY_EINVAL;
    }
    c->nnodes = nn;
    int64_t cn = T.cap_nodes;
    GROW(T.geo, nn, cn);
    GROW(T.thin, nn, cn);
    GROW(T.thick, nn, cn);
    GROW(T.prefix, nn, cn);
    GROW(T.mom, 11 * nn, cn * 11);
    T.cap_nodes = std::max(T.cap_nodes, nn);
#undef GROW

    TR_CUDA(cudaMemsetAsync(c->dt.err, 0, sizeof(unsigned), st));
    TR_CUDA(cudaMemsetAsync(T.geo, 0xff, sizeof(int4) * nn, st));
    TR_CUDA(cudaMemsetAsync(T.leaf_node, 0xff, sizeof(int32_t) * N, st));
    for (int l = lmax; l >= 0; --l) {
        LevelArgs a{T.keys, T.prefix, T.geo, T.leaf_node, lmax, l, c->level_off[l],
                    l < lmax ? c->level_off[l + 1] : 0, nint[l], nleaf[l], llo[l]};
        if (nint[l] > 0) {
            k_level_internal<<<nblk(nint[l], 256), 256, 0, st>>>(a);
            ++c->launches;
        }
        if (nleaf[l] > 0) {
            k_level_leaves<<<nblk(nleaf[l], 256), 256, 0, st>>>(a);
            ++c->launches;
        }
    }
    for (int l = 0; l <= lmax; ++l)
        if (nent[l] > 0) {
            k_check_nodes<<<nblk(nent[l], 256), 256, 0, st>>>(
                T.prefix, T.geo, T.leaf_node, c->level_off[l], nent[l],
                l < lmax ? c->level_off[l + 1] : 0, l < lmax ? nent[l + 1] : 0, N, c->dt.err);
            ++c->launches;
        }
    k_check_leaves<<<nblk(N, 256), 256, 0, st>>>(T.leaf_node, N, nn, c->dt.err);
    ++c->launches;
    {
        unsigned herr0 = 0;
        TR_CUDA(cudaGetLastError());
        TR_CUDA(cudaMemcpyAsync(&herr0, c->dt.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaStreamSynchronize(st));
        if (herr0) {
            TR_CUDA(cudaMemsetAsync(c->dt.err, 0, sizeof(unsigned), st));
            set_error("grid: leaves do not form a complete octree (overlapping or missing cells)");
            return TREERAY_EINVAL;
        }
    }

    // ---- moments
    MomArgs m{lg, T.perm, T.leaf_node, rho, Td, kappa, dstars, n_stars, gr->box,
              c->p.kappa_model, c->p.kappa0, c->p.kappa_ext_scale, c->p.dust_emission, nn, N,
              T.mom, T.geo, T.kap, T.tau, T.jsrc, T.psrc, T.thickflag, T.rho,
              kappa ? T.kin : nullptr, nullptr, c->dt.err};
    k_leaf_moments<<<nblk(N, 128), 128, 0, st>>>(m);
    ++c->launches;
    for (int l = lmax - 1; l >= 0; --l)
        if (nent[l] > 0) {
            k_internal_moments<<<nblk(nent[l], 128), 128, 0, st>>>(T.geo, T.mom, nn, c->level_off[l],
                                                                   nent[l], nullptr);
            ++c->launches;
        }
    k_scale<<<1, 1, 0, st>>>(T.mom, nn, c->u, c->dt.scal, nullptr);
    ++c->launches;
    k_pack<<<nblk(nn, 256), 256, 0, st>>>(T.geo, T.mom, nn, c->u, c->dt.scal, T.thin, T.thick, nullptr);
    ++c->launches;
    TR_CUDA(cudaGetLastError());
    double root_vk = 0.0;
    unsigned herr = 0;
    TR_CUDA(cudaMemcpyAsync(&root_vk, T.mom + 5 * nn, sizeof(double), cudaMemcpyDeviceToHost, st));
    TR_CUDA(cudaMemcpyAsync(&herr, c->dt.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    TR_CUDA(cudaStreamSynchronize(st));
    if (herr & kErrOctree) {
        set_error("grid: leaves do not form a complete octree");
        return TREERAY_EINVAL;
    }
    if (herr & kErrInput) {
        // reported here; the bit is cleared so that a later build on valid inputs succeeds
        const unsigned rest = herr & ~(unsigned)kErrInput;
        TR_CUDA(cudaMemcpy(c->dt.err, &rest, sizeof(unsigned), cudaMemcpyHostToDevice));
        set_error("rho, Td and kappa must be finite and >= 0");
        return TREERAY_EINVAL;
    }
    c->has_thick = root_vk > 0.0;
    c->grid_n = gr->n;
    c->n_stars = n_stars;
    c->kin_given = kappa != nullptr;
    const treeray_status rt = upload_tables(c, st);
    if (rt == TREERAY_OK) apply_cached_launch_choice(c);
    return rt;
}

// New dust temperatures on the same grid, densities, opacities and stars: leaf
// quantities, node moments, the luminosity scale and the walk records are recomputed;
// keys, structure and tables are kept. No host synchronisation, so the sequence can be
// captured in a CUDA graph. With skip != nullptr every kernel returns at once while
// *skip != 0 (the fixed point has converged).
treeray_status refresh_tree(treeray_ctx* c, const float* Td, const int* skip, cudaStream_t st) {
    DeviceTree& T = c->tree;
    const int64_t N = c->nleaves, nn = c->nnodes;
    LeafGrid lg{c->amr ? 0 : c->grid_n, c->lmax, T.blocks};
    MomArgs m{lg, T.perm, T.leaf_node, T.rho, Td, c->kin_given ? T.kin : nullptr, T.stars, c->n_stars,
              c->box, c->p.kappa_model, c->p.kappa0, c->p.kappa_ext_scale, c->p.dust_emission, nn, N,
              T.mom, T.geo, T.kap, T.tau, T.jsrc, T.psrc, T.thickflag, T.rho, nullptr, skip, c->dt.err};
    k_leaf_moments<<<nblk(N, 128), 128, 0, st>>>(m);
    ++c->launches;
    for (int l = c->lmax - 1; l >= 0; --l)
        if (c->level_cnt[l] > 0) {
            k_internal_moments<<<nblk(c->level_cnt[l], 128), 128, 0, st>>>(T.geo, T.mom, nn, c->level_off[l],
                                                                           c->level_cnt[l], skip);
            ++c->launches;
        }
    k_scale<<<1, 1, 0, st>>>(T.mom, nn, c->u, c->dt.scal, skip);
    ++c->launches;
    k_pack<<<nblk(nn, 256), 256, 0, st>>>(T.geo, T.mom, nn, c->u, c->dt.scal, T.thin, T.thick, skip);
    ++c->launches;
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}

}  // namespace tr
