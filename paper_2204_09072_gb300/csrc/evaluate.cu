// Ray evaluation (Secs. 4.2-4.4 of Klepitko et al. 2023): a team of warps per target.
//
// Walk: a stack of child groups (the 8 sub-nodes of an opened node are contiguous). Each
// step the team pops up to 4 groups per warp, so every thread tests one node; opened
// nodes push their child group through a ballot compaction. Open/accept, the segment
// index, the angular-kernel key and straddled segment boundaries are decided in exact
// integer arithmetic on the squared centre distance (thresholds built on the host in FP64).
//
// Deposit (Secs. 4.2.1-4.2.2): per (segment i, ray h) accumulators in the team's slice of
// global memory, added to by reductions in L2
//   thin:  L^ += a b L,  A^ += a b A~          (b = R_i^2 / r_COL^2, a = alpha_node(h))
//   thick: L^ += a L_V,  A^ += A~,  V^ += a V,  Q^ += a b V, plus straddle flags.
// Integration (Sec. 4.3): segments inside out per ray in FP32, the transmission carried as
// a product of per-segment e^-tau and the flux sums as float pairs (error-free
// transformations), so the GB300's slow FP64 pipe is not on the path. Finalization
// (Sec. 4.4): J = sum_h F^h / 4 pi, F = -sum_h F^h n^h, converted to CGS in FP64.
//
// Internal units: lengths in half-cells of the finest level (u cm), luminosities in
// L_scale erg/s; fluxes come out in L_scale / u^2 and are converted to CGS at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "internal.h"

namespace tr {

struct __align__(16) EvalArgs {
    const int4* __restrict__ geo;
    const float4* __restrict__ thin;
    const float4* __restrict__ thick;
    const int32_t* __restrict__ leaf_node;
    const int32_t* __restrict__ perm;
    const int32_t* __restrict__ inv_perm;
    const int32_t* __restrict__ targets;
    const double* __restrict__ jsrc;
    const float* __restrict__ nhat;     // [orientations][npix][3]
    const int32_t* __restrict__ aoff;   // [orientations][aoff_stride]
    const int2* __restrict__ apair;     // [orientations][aoff_stride - 1] (first entry, end)
    const uint32_t* __restrict__ aent;
    const uint8_t* __restrict__ orient;  // per leaf (caller order): its ray orientation, or null
    int64_t aoff_stride;
    const int64_t* __restrict__ bin_thr;
    const longlong2* __restrict__ bin_thr2;  // (thr[i], thr[i+1]) side by side
    const float* __restrict__ R2;
    const float* __restrict__ Rh;       // [target level][nbins] R_i (half-cells)
    const double* __restrict__ Rd;      // [target level][nbins] R_i in FP64 (COL decisions)
    const double* __restrict__ mom;     // FP64 node moments [11][nn] (COL in rows 8..10)
    int64_t nn;
    const int64_t* __restrict__ open_max;
    const int64_t* __restrict__ str_lo;
    const int64_t* __restrict__ str_hi;
    const float2* __restrict__ lvlp;    // per target level: segment-guess parameters
    const double* __restrict__ scal;
    unsigned* err;
    unsigned long long* queue;
    float* J;
    double* F;
    float* tau_mean;   // optional: mean over rays of the ray optical depth
    float* tau_min;    // optional: smallest ray optical depth
    int32_t* acc_counts;   // accepted-list mode
    int32_t* acc_ids;
    unsigned long long* stats;  // accepted-list mode: totals of visits, accepted, entries
    const int* skip;            // fixed-point mode: return at once when *skip != 0
    int* stack;                 // team stacks: stack_cap ints per block of the launch
    float* gtile;               // the teams' (segment x ray) tiles in global memory
    int64_t gtile_stride;       // floats per team in gtile (tile, then merge flags)
    int acc_cap;
    int64_t n;
    int64_t nleaves;
    int lmax, nbins, D, stack_cap, npix;
    int periodic;     // bit a: axis a periodic (closest copies)
    int col_mapping;  // map accepted nodes at their centre of luminosity
    float inv_s3;  // 1 / alpha_s^3: weight of one sub-cube sample of the angular kernel
    double u;
    double inv_u2;  // 1 / u^2: flux unit = L_scale / u^2 (L_scale a power of two)
};

// A batch launch's parameters: the launch-wide fields (work counter, total targets, team
// stacks) in `launch`, then up to kMaxLaunchBoxes box descriptors and the first target
// of each box; a batch with more boxes is launched in chunks. Sized to fit the 32764
// bytes of kernel parameters.
constexpr int kMaxLaunchBoxes = (32764 - (int)sizeof(EvalArgs) - 16) / ((int)sizeof(EvalArgs) + 8) - 1;
struct __align__(16) BatchArgs {
    EvalArgs launch;
    EvalArgs box[kMaxLaunchBoxes];
    int64_t start[kMaxLaunchBoxes + 1];
    int nbox;
};
static_assert(sizeof(BatchArgs) <= 32764, "batch parameters exceed the kernel parameter space");

namespace {


__device__ __forceinline__ int alpha_key(int o, int elog) {
    // K = 8 o / E when integral, else the nearest odd integer (floor(4 o / E) * 2 + 1)
    const int e = 8 * o;
    if ((e & ((1 << elog) - 1)) == 0) return e >> elog;
    return 2 * ((4 * o) >> elog) + 1;
}

// Largest j in [1, nb-1] with d2 >= arr[j] (arr non-decreasing), else 0, starting from a
// guess: the fix-up loops make the result exact whatever the guess.
// The same on the threshold pairs (thr[i], thr[i+1]) of one level: a correct guess costs one
// 16-byte load.
__device__ __forceinline__ int fixup_pair(int g, int64_t d2, const longlong2* __restrict__ pr, int nb) {
    g = max(0, min(g, nb - 1));
    const longlong2 t = __ldg(pr + g);
    if (d2 >= t.y) {
        do ++g;
        while (g + 1 < nb && d2 >= __ldg(pr + g).y);
    } else if (g > 0 && d2 < t.x) {
        do --g;
        while (g > 0 && d2 < __ldg(pr + g).x);
    }
    return g;
}
__device__ __forceinline__ int fixup(int g, int64_t d2, const int64_t* __restrict__ arr, int nb) {
    g = max(0, min(g, nb - 1));
    while (g + 1 < nb && d2 >= __ldg(arr + g + 1)) ++g;
    while (g > 0 && d2 < __ldg(arr + g)) --g;
    return g;
}

// Guess of the segment holding squared distance x2 for a target level (the integer
// thresholds then decide): geometric radii, lp = (1 / R_0^2, 0.5 / log2 g), gives
// 0.5 log2(x2 / R_0^2) / log2(g); quadratic radii, lp = (-R_0, nb^2 / (R_max - R_0)),
// give sqrt((d - R_0) nb^2 / (R_max - R_0)).
__device__ __forceinline__ int guess_bin(float x2, float2 lp) {
    if (lp.x < 0.0f)  // quadratic radii: lp = (-R_0, nb^2 / (R_max - R_0))
        return x2 > 0.0f ? (int)sqrtf(fmaxf(sqrtf(x2) + lp.x, 0.0f) * lp.y) : 0;
    return x2 > 0.0f ? (int)(__log2f(x2 * lp.x) * lp.y) : 0;  // geometric radii
}

// Exact integer -> float conversions on the FP32 and integer pipes: the integer is
// placed in the mantissa of a float whose unit in the last place is 1.
__device__ __forceinline__ float small_int_to_float(int v) {  // exact for |v| < 2^22
    return __int_as_float(0x4B400000 + v) - 12582912.0f;
}
__device__ __forceinline__ float count_to_float(uint32_t v) {  // exact for v < 2^23
    return __uint_as_float(0x4B000000u | v) - 8388608.0f;
}

// Largest j in [1, nb-1] with x2 >= R2[j] (R2 = R_j^2 in FP32), else 0.
__device__ __forceinline__ int fixup_r2(int g, float x2, const float* __restrict__ R2, int nb) {
    g = max(0, min(g, nb - 1));
    while (g + 1 < nb && x2 >= __ldg(R2 + g + 1)) ++g;
    while (g > 0 && x2 < __ldg(R2 + g)) --g;
    return g;
}
// Squared length in FP32, evaluated in a fixed order and never fused, as the oracle does.
__device__ __forceinline__ float sq3_rn(float x, float y, float z) {
    return __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z));
}

// Mapping decisions of a node taken at its centre of luminosity (Sec. 7.6): segment i,
// angular key K and, for thick material, the straddled segment boundaries [ilo, ihi).
// They are defined on the COL position p = q + (COL - centre) in FP64: i is the largest j
// with |p|^2 >= R_j^2, |p|^2 = (p_x^2 + p_y^2) + p_z^2; K = 2 floor(4 p / E) + 1 per axis;
// a boundary j is straddled from below when |p|^2 >= (R_j + s)^2 and from above when
// R_j <= s or |p|^2 >= (R_j - s)^2, s = sqrt(3)/2 E. The FP32 position (the node record's
// COL offset) decides wherever it lies farther from every threshold than 2^-20 of the
// compared magnitudes, which bounds its few FP32 roundings many times over; a node closer
// to a threshold is decided from the FP64 COL of its moments, in FP64 as defined.
struct ColMap {
    int i, kx, ky, kz, ilo, ihi;
};
constexpr float kColTol = 9.5367431640625e-07f;  // 2^-20

__device__ __noinline__ ColMap col_decide_fp64(const EvalArgs& A, int node, int qx, int qy, int qz, int lvl,
                                               int tl, bool straddle) {
    ColMap m{0, 0, 0, 0, 0, 0};
    const int nb = A.nbins;
    const double* Rd = A.Rd + (int64_t)tl * nb;
    const int4 g = __ldg(A.geo + node);
    const double px = __dadd_rn((double)qx, __dsub_rn(__ldg(A.mom + 8 * A.nn + node), (double)g.x));
    const double py = __dadd_rn((double)qy, __dsub_rn(__ldg(A.mom + 9 * A.nn + node), (double)g.y));
    const double pz = __dadd_rn((double)qz, __dsub_rn(__ldg(A.mom + 10 * A.nn + node), (double)(g.z & 0xffffff)));
    const double pd2 = __dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz));
    for (int j = 1; j < nb; ++j) {
        const double R = __ldg(Rd + j);
        if (pd2 >= __dmul_rn(R, R)) m.i = j;
    }
    const double E = (double)(2 << (A.lmax - lvl));
    m.kx = 2 * (int)floor(__ddiv_rn(__dmul_rn(4.0, px), E)) + 1;
    m.ky = 2 * (int)floor(__ddiv_rn(__dmul_rn(4.0, py), E)) + 1;
    m.kz = 2 * (int)floor(__ddiv_rn(__dmul_rn(4.0, pz), E)) + 1;
    if (straddle) {
        const double sd = __dmul_rn(__dmul_rn(sqrt(3.0), 0.5), E);
        for (int j = 1; j < nb; ++j) {
            const double R = __ldg(Rd + j);
            const double up = __dadd_rn(R, sd), dn = __dsub_rn(R, sd);
            if (pd2 >= __dmul_rn(up, up)) m.ilo = j;
            if (dn <= 0.0 || pd2 >= __dmul_rn(dn, dn)) m.ihi = j;
        }
    }
    return m;
}

// The same decisions from the FP32 record (c: the COL offset held in the node record), with
// the FP64 path where the FP32 position is too close to a threshold. (rx, ry, rz) = q + c in
// FP32, as the radial kernel uses it.
__device__ __forceinline__ ColMap col_decide(const EvalArgs& A, int node, int qx, int qy, int qz, float rx,
                                             float ry, float rz, int lvl, int tl, float2 lp, bool straddle) {
    ColMap m;
    const int nb = A.nbins;
    const float* R2 = A.R2 + (int64_t)tl * nb;
    const float pd2 = sq3_rn(rx, ry, rz);
    const float Ef = (float)(2 << (A.lmax - lvl));
    const float tol = kColTol * (pd2 + Ef * Ef);
    m.i = fixup_r2(guess_bin(pd2, lp), pd2, R2, nb);
    bool unsure = (m.i > 0 && pd2 - __ldg(R2 + m.i) <= tol) || (m.i + 1 < nb && __ldg(R2 + m.i + 1) - pd2 <= tol);
    const float sc = ldexpf(1.0f, 1 - (A.lmax - lvl));  // 4 / E
    const float tx = rx * sc, ty = ry * sc, tz = rz * sc;
    const float fx = floorf(tx), fy = floorf(ty), fz = floorf(tz);
    unsure = unsure || tx - fx <= kColTol * (fabsf(tx) + 1.0f) || fx + 1.0f - tx <= kColTol * (fabsf(tx) + 1.0f) ||
             ty - fy <= kColTol * (fabsf(ty) + 1.0f) || fy + 1.0f - ty <= kColTol * (fabsf(ty) + 1.0f) ||
             tz - fz <= kColTol * (fabsf(tz) + 1.0f) || fz + 1.0f - tz <= kColTol * (fabsf(tz) + 1.0f);
    m.kx = 2 * (int)fx + 1;
    m.ky = 2 * (int)fy + 1;
    m.kz = 2 * (int)fz + 1;
    m.ilo = 0;
    m.ihi = 0;
    if (straddle) {
        const float* Rh = A.Rh + (int64_t)tl * nb;
        const float sd = 0.8660254f * Ef;
        for (int j = 1; j < nb; ++j) {
            const float R = __ldg(Rh + j);
            const float up = R + sd, dn = R - sd;
            const float u2 = up * up, d2f = dn * dn;
            if (fabsf(pd2 - u2) <= kColTol * (pd2 + u2) || fabsf(dn) <= kColTol * up ||
                (dn > 0.0f && fabsf(pd2 - d2f) <= kColTol * (pd2 + d2f)))
                unsure = true;
            if (pd2 >= u2) m.ilo = j;
            if (dn <= 0.0f || pd2 >= d2f) m.ihi = j;
        }
    }
    if (unsure) return col_decide_fp64(A, node, qx, qy, qz, lvl, tl, straddle);
    return m;
}

// Closest periodic copy on one axis (Sec. 4.2): the offset o (half-cells) is brought into
// [-half, half], half = half the box; an offset of exactly +-half has two closest copies
// and sets `bit` in `ties`.
__device__ __forceinline__ int closest_copy(int o, int half, int bit, int& ties) {
    if (o > half) o -= 2 * half;
    else if (o < -half) o += 2 * half;
    if (o == half || o == -half) ties |= bit;
    return o;
}
__device__ __forceinline__ int copy_offset(int o, int ties, int bit, int m, int half) {
    return (ties & bit) ? ((m & bit) ? half : -half) : o;
}

// Error-free transformations (Knuth's TwoSum; the FMA residual of a product), written
// with the _rn intrinsics so that the compiler never fuses them. An unevaluated pair
// (hi, lo) then carries about 48 significant bits through FP32 arithmetic.
__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float b) {
    const float s = __fadd_rn(hi, b);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}
__device__ __forceinline__ void add_product(float& hi, float& lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);  // a b - p exactly
    two_sum_into(hi, lo, p);
    lo = __fadd_rn(lo, e);
}
__device__ __forceinline__ void add_pair(float& hi, float& lo, float bh, float bl) {
    two_sum_into(hi, lo, bh);
    lo = __fadd_rn(lo, bl);
}

// Accepted-list / walk-statistics mode: the walk alone, one warp per target.
__global__ void __launch_bounds__(256) k_walk_list(EvalArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* stack = reinterpret_cast<int*>(smem) + (size_t)warp * a.stack_cap;
    const unsigned full = 0xffffffffu;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int W = 2 * a.D + 1;
    for (;;) {
        long long q = 0;
        if (lane == 0) q = (long long)atomicAdd(a.queue, 1ull);
        q = __shfl_sync(full, q, 0);
        if (q >= a.n) break;
        int64_t s, cell;
        if (a.targets) {
            const int32_t k = a.targets[q];
            if (k < 0 || k >= a.nleaves) {
                if (lane == 0) atomicOr(a.err, kErrTarget);
                continue;
            }
            s = a.inv_perm[k];
            cell = k;
        } else {
            s = q;
            cell = a.perm[s];
        }
        // angular-kernel table of the target's ray orientation
        const int32_t* aoff = a.aoff + (a.orient ? (int64_t)a.orient[cell] * a.aoff_stride : 0);
        const int4 tg = a.geo[a.leaf_node[s]];
        const int tx = tg.x, ty = tg.y, tz = tg.z & 0xffffff;
        int nacc = 0;
        long long nvis = 0, nent = 0;
        int sp = 0;
        const int4 root = a.geo[0];
        if (root.w >= 0) {
            if (lane == 0) stack[0] = root.w;
            sp = 1;
        }
        bool overflow = false;
        __syncwarp();
        while (sp > 0) {
            const int ng = sp < 4 ? sp : 4;
            const int g = lane >> 3;
            const bool valid = g < ng;
            const int node = valid ? stack[sp - ng + g] + (lane & 7) : 0;
            __syncwarp();
            sp -= ng;
            bool open = false, acc = false;
            int4 gg = make_int4(0, 0, 0, 0);
            int ox = 0, oy = 0, oz = 0, lvl = 0;
            int64_t d2 = 0;
            int ties = 0;
            if (valid) {
                gg = __ldg(a.geo + node);
                lvl = gg.z >> 24;
                ox = gg.x - tx;
                oy = gg.y - ty;
                oz = (gg.z & 0xffffff) - tz;
                if (a.periodic) {
                    const int half = 1 << a.lmax;
                    if (a.periodic & 1) ox = closest_copy(ox, half, 1, ties);
                    if (a.periodic & 2) oy = closest_copy(oy, half, 2, ties);
                    if (a.periodic & 4) oz = closest_copy(oz, half, 4, ties);
                }
                d2 = (int64_t)ox * ox + (int64_t)oy * oy + (int64_t)oz * oz;
                if (gg.w >= 0) {
                    const int E = 2 << (a.lmax - lvl);
                    const bool inside = 2 * abs(ox) < E && 2 * abs(oy) < E && 2 * abs(oz) < E;
                    open = inside || d2 <= __ldg(a.open_max + lvl);
                }
                acc = !open;
            }
            const unsigned om = __ballot_sync(full, open);
            if (open) {
                const int pos = sp + __popc(om & lt_mask);
                if (pos < a.stack_cap) stack[pos] = gg.w;
            }
            sp += __popc(om);
            if (sp > a.stack_cap) {
                overflow = true;
                break;
            }
            const unsigned am = __ballot_sync(full, acc);
            if (acc && a.acc_ids) {
                const int pos = nacc + __popc(am & lt_mask);
                if (pos < a.acc_cap) a.acc_ids[q * (int64_t)a.acc_cap + pos] = node;
            }
            nacc += __popc(am);
            nvis += __popc(__ballot_sync(full, valid));
            if (a.stats && acc && d2 != 0) {
                const int elog = a.lmax - lvl + 1;
                const int half = 1 << a.lmax;
                float cx = 0.0f, cy = 0.0f, cz = 0.0f;  // COL offset when nodes map at their COL
                if (a.col_mapping) {
                    const float4 v0 = __ldg(a.thin + node);
                    cx = v0.z;
                    cy = v0.w;
                    cz = __ldg(a.thick + node).x;
                }
                const bool colmap = cx != 0.0f || cy != 0.0f || cz != 0.0f;
                const int tl = tg.z >> 24;
                for (int m = 0; m < 8; ++m) {  // entries of every closest copy
                    if (m & ~ties) continue;
                    const int qx = copy_offset(ox, ties, 1, m, half), qy = copy_offset(oy, ties, 2, m, half),
                              qz = copy_offset(oz, ties, 4, m, half);
                    int Kx, Ky, Kz;
                    if (colmap) {
                        const ColMap cm = col_decide(a, node, qx, qy, qz, small_int_to_float(qx) + cx,
                                                     small_int_to_float(qy) + cy, small_int_to_float(qz) + cz, lvl,
                                                     tl, __ldg(a.lvlp + tl), false);
                        Kx = cm.kx;
                        Ky = cm.ky;
                        Kz = cm.kz;
                    } else {
                        Kx = alpha_key(qx, elog);
                        Ky = alpha_key(qy, elog);
                        Kz = alpha_key(qz, elog);
                    }
                    if (abs(Kx) <= a.D && abs(Ky) <= a.D && abs(Kz) <= a.D) {
                        const int idx = ((Kz + a.D) * W + (Ky + a.D)) * W + (Kx + a.D);
                        nent += __ldg(aoff + idx + 1) - __ldg(aoff + idx);
                    }
                }
            }
        }
        overflow = __any_sync(full, overflow);
        if (overflow) {
            if (lane == 0) atomicOr(a.err, kErrStack);
            continue;
        }
        if (a.acc_counts && lane == 0) a.acc_counts[q] = nacc;
        if (a.stats) {
            for (int off = 16; off > 0; off >>= 1) nent += __shfl_xor_sync(full, nent, off);
            if (lane == 0) {
                atomicAdd(a.stats + 0, (unsigned long long)(nvis + 1));
                atomicAdd(a.stats + 1, (unsigned long long)nacc + (root.w >= 0 ? 0ull : 1ull));
                atomicAdd(a.stats + 2, (unsigned long long)nent);
            }
        }
        __syncwarp();
    }
}

// entries per warp and walk step spread one per lane (more go through a serial fallback)
__host__ __device__ constexpr int owner_cap(bool thick) { return thick ? 160 : 256; }

// Where a team's (segment x ray) tile lives. On sm_103a an FP32 addition to shared memory is
// a compare-and-swap loop through the SM's load/store data pipe, while an FP32 reduction to
// global memory (red.global.add.f32) is native in L2 and costs the SM one fire-and-forget
// request. So every team keeps its tile in its own slice of global memory (L2-resident: the
// slices of one launch take 20-60 MB at 48 rays) and reads it back through L2
// (ld.global.cg) after the team barrier. Each cell's thin L^ and A^ are interleaved, so that
// one vector reduction (red.global.add.v2.f32) deposits both; the four thick quantities keep
// an array each (interleaving them into one vector reduction measured slower at 48 rays).
// 768 rays (N_side 8): owner bytes for 2048 entries per warp pass, no batches
template <int NPIX>
struct WideRays {
    static constexpr bool on = NPIX > 192;
};
__host__ __device__ constexpr int owner_cap_for(int npix, bool thick) { return npix > 192 ? 2048 : owner_cap(thick); }
__device__ __forceinline__ float gld(const float* p) { return __ldcg(p); }
__device__ __forceinline__ void gst(float* p, float v) { __stcg(p, v); }
// p[0] += a, p[1] += b in L2 (p 8-byte aligned), one request
__device__ __forceinline__ void red_add_v2(float* p, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}
// thin deposit of cell c: L^ += l, A^ += ar (one interleaved pair; tA = tL + 1)
__device__ __forceinline__ void deposit_thin(float* tL, int c, float l, float ar) { red_add_v2(tL + 2 * c, l, ar); }
__device__ __forceinline__ unsigned long long gld64(const unsigned long long* p) { return __ldcg(p); }
__device__ __forceinline__ void gst64(unsigned long long* p, unsigned long long v) { __stcg(p, v); }

// Row stride of the (segment x ray) tile, in cells. Thin tiles: 4 cells more than the rays
// (128^3 cloud at 48 rays: 42.3 ms against 42.5 unpadded; 192 rays: 69.2 against 68.6).
// Thick tiles are not padded (a smaller footprint in L2: collapsing core 76.6 -> 74.6 ms
// against one word more).
__host__ __device__ constexpr int tile_row(int npix, bool thick) { return npix + (thick ? 0 : 4); }
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Warps resident per SM that the register budget is cut for: with the FP32 tiles in global
// memory no kernel is limited by shared memory, and a full SM (64 warps, 32 registers with
// a few spills) measured fastest for thin and thick tiles alike (collapsing core, thick:
// 103.6 ms at 36 warps, 93.3 at 48, 76.6 at 64).
constexpr int min_warps_per_sm(int, bool) { return 64; }

// Deposit of an accepted node whose closest periodic copies are tied (it lies exactly half
// a box away on a periodic axis): every closest copy, with weight 1/2 per tied axis, by the
// node's own thread with atomics. The copies share |offset| per axis, hence
// d^2, the segment and the straddled boundaries; alpha and beta differ. Such nodes lie on
// the planes half a box from the target, so this path is rare.
template <int NPIX, bool THICK>
__device__ __noinline__ void deposit_tied_copies(const EvalArgs& A, const int32_t* aoff, float* tL, float* tA,
                                                 float* tLk, float* tAk,
                                                 float* tVk, float* tQk, unsigned long long* flags, int node,
                                                 int ox, int oy, int oz, int ties, int lvl, int64_t d2, int tl,
                                                 float2 lp) {
    const int nb = A.nbins;
    const int64_t* thr = A.bin_thr + (int64_t)tl * nb;
    const float* R2 = A.R2 + (int64_t)tl * nb;
    const int64_t* lo = A.str_lo + ((int64_t)tl * (A.lmax + 1) + lvl) * nb;
    const int64_t* hi = A.str_hi + ((int64_t)tl * (A.lmax + 1) + lvl) * nb;
    const int W = 2 * A.D + 1;
    const int half = 1 << A.lmax;
    const float inv_s3 = A.inv_s3;
    const float wt = 1.0f / (float)(1 << __popc(ties));
    const float4 v0 = __ldg(A.thin + node);
    const float4 v1 = __ldg(A.thick + node);
    const bool thick = THICK && v1.w > 0.0f;
    const bool colmap = A.col_mapping && (v0.z != 0.0f || v0.w != 0.0f || v1.x != 0.0f);
    const float sd = 0.8660254f * (float)(2 << (A.lmax - lvl));
    // at the geometric centre the copies share |offset| per axis, hence d^2, the segment
    // and the straddled boundaries; at the COL each copy has its own
    const float fd2 = (float)d2;
    const int i0 = fixup(guess_bin(fd2, lp), d2, thr, nb);
    unsigned long long fmask0 = 0ull;
    if (thick && !colmap) {
        const float d = sqrtf(fd2);
        const float dl = fmaxf(d - sd, 0.0f), dh = d + sd;
        const int ilo = fixup(guess_bin(dl * dl, lp), d2, lo, nb);
        const int ihi = fixup(guess_bin(dh * dh, lp), d2, hi, nb);
        for (int j = ilo; j < ihi; ++j) fmask0 |= 1ull << j;
    }
    const int elog = A.lmax - lvl + 1;
    for (int m = 0; m < 8; ++m) {
        if (m & ~ties) continue;
        const int qx = copy_offset(ox, ties, 1, m, half), qy = copy_offset(oy, ties, 2, m, half),
                  qz = copy_offset(oz, ties, 4, m, half);
        const float rx = small_int_to_float(qx) + v0.z, ry = small_int_to_float(qy) + v0.w,
                    rz = small_int_to_float(qz) + v1.x;
        int i = i0;
        unsigned long long fmask = fmask0;
        int Kx = alpha_key(qx, elog), Ky = alpha_key(qy, elog), Kz = alpha_key(qz, elog);
        if (colmap) {
            const ColMap cm = col_decide(A, node, qx, qy, qz, rx, ry, rz, lvl, tl, lp, thick);
            i = cm.i;
            Kx = cm.kx;
            Ky = cm.ky;
            Kz = cm.kz;
            if (thick) {
                fmask = 0ull;
                for (int j = cm.ilo; j < cm.ihi; ++j) fmask |= 1ull << j;
            }
        }
        const float beta = __ldg(R2 + i) / (rx * rx + ry * ry + rz * rz);
        if (abs(Kx) > A.D || abs(Ky) > A.D || abs(Kz) > A.D) {
            atomicOr(A.err, kErrAlphaKey);
            continue;
        }
        const int idx = ((Kz + A.D) * W + (Ky + A.D)) * W + (Kx + A.D);
        const int e0 = __ldg(aoff + idx), e1 = __ldg(aoff + idx + 1);
        if (e1 == e0) atomicOr(A.err, kErrAlphaKey);
        const float bL = beta * v0.x * inv_s3 * wt, bA = beta * v0.y * inv_s3 * wt;
        for (int e = e0; e < e1; ++e) {
            const uint32_t ent = __ldg(A.aent + e);
            const int h = (int)(ent & 0xffffu);
            const int c = i * tile_row(NPIX, THICK) + h;
            const float w = count_to_float(ent >> 16);
            deposit_thin(tL, c, w * bL, w * bA);
            if (thick) {
                const float wn = w * inv_s3;
                atomicAdd(tLk + c, wn * v1.y * wt);
                atomicAdd(tAk + c, v1.z * wt);
                atomicAdd(tVk + c, wn * v1.w * wt);
                atomicAdd(tQk + c, wn * beta * v1.w * wt);
                if (fmask) atomicOr(flags + h, fmask);
            }
        }
    }
}

// Evaluation kernel: a team of WPT warps per target shares one walk stack (its block's
// slice of a global scratch array, L1-resident) and one (segment x ray) tile (its block's
// slice of another, L2-resident); the block processes one target at a time and takes the
// next from a global work counter (persistent grid).
//   walk:    each step the team pops up to 4 WPT child groups (32 WPT nodes), tests them,
//            appends the opened nodes' child groups to the stack (one shared-memory
//            atomic per warp) and maps the accepted ones (segment, beta, angular key);
//   deposit: the warp's thin deposits are spread one angular-kernel entry per lane, in
//            child-major node order so that sibling nodes, which often hit the same cell,
//            fall into different rounds; one L2 vector reduction of the cell's (L^, A^)
//            pair per entry; thick deposits follow in a second pass, also one entry per
//            lane;
//   rays:    threads integrate the rays' segments inside out (thin tiles with spare
//            threads cut each ray into consecutive parts joined by their transmission),
//            then the team reduces J and F.
// BATCH: the targets of several boxes share the work counter, each box with its own
// descriptor. Either way the descriptors are kernel parameters, read from the constant
// bank: one box's as the launch's own, a batch's as an array (BatchArgs).
template <int NPIX, bool THICK, int WPT, bool GENERAL, bool BATCH>
__device__ __forceinline__ void evaluate_team(const EvalArgs& a, const BatchArgs* bp) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NT = WPT * 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = a.nbins;
    constexpr int ROW = tile_row(NPIX, THICK);
    const int cells = nb * ROW;
    // layout of the team's slice of global memory (16-byte aligned parts):
    //   thin (L^, A^) pairs [nb][ROW][2] f32 | THICK: L^, A^, V^, Q^ thick [nb][ROW] f32
    //   each, then the merge flags [NPIX] u64
    // shared memory: per warp entry owners u8[owner_cap]
    // The team's stack of child groups is this block's slice of a global scratch array:
    // it stays in L1, and leaving it out of shared memory lets more teams share an SM.
    constexpr int nq = THICK ? 6 : 2;
    constexpr int LS = 2;  // stride of a cell's L^ and A^ (interleaved)
    float* tL = a.gtile + (size_t)blockIdx.x * a.gtile_stride;
    float* tA = tL + 1;
    float* tLk = tL + 2 * cells;  // thick tiles only
    float* tAk = tLk + cells;
    float* tVk = tAk + cells;
    float* tQk = tVk + cells;
    unsigned long long* flags =
        reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(tL) + align16((size_t)nq * cells * 4));
    // each entry's node data comes from the owner lane by shuffles (fewer shared-memory
    // operations and registers than a per-warp node buffer)
    constexpr int OCAP = owner_cap_for(NPIX, THICK);
    unsigned char* owner = smem + warp * OCAP;
    const int stack_cap = a.stack_cap;
    int* stack = a.stack + (size_t)blockIdx.x * stack_cap;
    __shared__ int s_sp, s_overflow;
    __shared__ long long s_q;
    __shared__ const int32_t* s_aoff;  // the target's orientation: angular-kernel table
    __shared__ const int2* s_apair;
    __shared__ const float* s_nhat;    // and ray directions
    __shared__ float s_red[7][WPT];  // J, then (hi, lo) pairs of F_x, F_y, F_z
    __shared__ float s_tau[2][WPT];
    const unsigned full = 0xffffffffu;
    const unsigned lt_mask = (1u << lane) - 1u;
    const float omega = (float)(4.0 * kPi / NPIX);
    if (a.skip && *a.skip) return;
    __shared__ int s_b;  // batch: the box of the current target

    for (;;) {
        if (tid == 0) s_q = (long long)atomicAdd(a.queue, 1ull);
        __syncthreads();
        long long q = s_q;
        if (q >= a.n) break;
        int b = 0;
        if constexpr (BATCH) {
            if (tid == 0) {
                int lo = 0, hi = bp->nbox - 1;  // last box with start[b] <= q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (bp->start[mid] <= q) lo = mid;
                    else hi = mid - 1;
                }
                s_b = lo;
            }
            __syncthreads();
            b = s_b;
            q -= bp->start[b];
        }
        __syncthreads();
        const EvalArgs& A = *(BATCH ? &bp->box[b] : &a);
        const int W = 2 * A.D + 1;
        const int4 root = A.geo[0];
        int64_t s;
        int64_t out, cell;
        if (A.targets) {
            const int32_t k = A.targets[q];
            if (k < 0 || k >= A.nleaves) {
                if (tid == 0) atomicOr(A.err, kErrTarget);
                __syncthreads();
                continue;
            }
            s = A.inv_perm[k];
            out = q;
            cell = k;
        } else {
            s = q;
            out = A.perm[s];
            cell = out;
        }
        const int tnode = A.leaf_node[s];
        const int4 tg = A.geo[tnode];
        const int tx = tg.x, ty = tg.y, tz = tg.z & 0xffffff;
        const int tl = tg.z >> 24;
        const longlong2* thr2 = A.bin_thr2 + (int64_t)tl * nb;
        const float* R2 = A.R2 + (int64_t)tl * nb;
        const float2 lp = __ldg(A.lvlp + tl);

        {  // zero the tile: 16-byte stores (it starts 16-byte aligned), then the tail
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            float4* g4 = reinterpret_cast<float4*>(tL);
            const int ng = nq * cells;
            for (int i = tid; i < ng / 4; i += NT) __stcg(g4 + i, z4);
            for (int i = (ng / 4) * 4 + tid; i < ng; i += NT) gst(tL + i, 0.0f);
        }
        if (THICK)
            for (int h = tid; h < NPIX; h += NT) gst64(flags + h, 0ull);
        if (tid == 0) {
            s_overflow = 0;
            s_sp = 0;
            if (root.w >= 0) {
                stack[0] = root.w;
                s_sp = 1;
            }
            const int o = A.orient ? (int)A.orient[cell] : 0;
            s_aoff = A.aoff + (int64_t)o * A.aoff_stride;
            s_apair = A.apair + (int64_t)o * (A.aoff_stride - 1);
            s_nhat = A.nhat + 3 * NPIX * o;
        }
        __syncthreads();
        for (;;) {
            const int sp = s_sp;
            if (sp == 0 || s_overflow) break;
            const int ng = sp < 4 * WPT ? sp : 4 * WPT;
            const int g = tid >> 3;
            const bool valid = g < ng;
            const int node = valid ? stack[sp - ng + g] + (tid & 7) : 0;
            __syncthreads();  // every pop is read before the stack is reused
            if (tid == 0) s_sp = sp - ng;
            __syncthreads();
            bool open = false, acc = false;
            int4 gg = make_int4(0, 0, 0, 0);
            int ox = 0, oy = 0, oz = 0, lvl = 0;
            int64_t d2 = 0;
            int ties = 0;
            if (valid) {
                gg = __ldg(A.geo + node);
                lvl = gg.z >> 24;
                ox = gg.x - tx;
                oy = gg.y - ty;
                oz = (gg.z & 0xffffff) - tz;
                if (GENERAL && A.periodic) {
                    const int half = 1 << A.lmax;
                    if (A.periodic & 1) ox = closest_copy(ox, half, 1, ties);
                    if (A.periodic & 2) oy = closest_copy(oy, half, 2, ties);
                    if (A.periodic & 4) oz = closest_copy(oz, half, 4, ties);
                }
                d2 = (int64_t)ox * ox + (int64_t)oy * oy + (int64_t)oz * oz;
                if (gg.w >= 0) {
                    const int E = 2 << (A.lmax - lvl);
                    const bool inside = 2 * abs(ox) < E && 2 * abs(oy) < E && 2 * abs(oz) < E;
                    open = inside || d2 <= __ldg(A.open_max + lvl);
                }
                acc = !open && d2 != 0;  // the own cell is deposited after the walk
            }
            const unsigned om = __ballot_sync(full, open);
            if (om) {
                int pos0 = 0;
                if (lane == 0) pos0 = atomicAdd(&s_sp, __popc(om));
                pos0 = __shfl_sync(full, pos0, 0);
                if (open) {
                    const int pos = pos0 + __popc(om & lt_mask);
                    if (pos < stack_cap) stack[pos] = gg.w;
                    else s_overflow = 1;
                }
            }
            // ---- map the accepted nodes onto the rays. Per node (one per thread): segment,
            // beta, angular-kernel key. The thin deposits of the warp's nodes are then
            // spread one angular-kernel entry per lane (a node's entries are distinct rays
            // of one segment), and the thick deposits after them in a second such pass.
            int ne = 0, ebase = 0, cbase = 0;
            float bL = 0.0f, bA = 0.0f;
            // thick deposits of this thread's node, spread over the warp after the thin ones:
            // entry count, the node's L_V, A~, V (thick record) and beta, merge flags
            int nk = 0;
            float kLV = 0.0f, kA = 0.0f, kV = 0.0f, kbeta = 0.0f;
            unsigned long long kfm = 0ull;
            if (GENERAL && acc && ties) {
                deposit_tied_copies<NPIX, THICK>(A, s_aoff, tL, tA, tLk, tAk, tVk, tQk, flags, node, ox, oy, oz,
                                                 ties, lvl, d2, tl, lp);
            } else if (acc) {
                // the float distance only guesses the segment; the integer d^2 decides it
                const float fx = small_int_to_float(ox), fy = small_int_to_float(oy), fz = small_int_to_float(oz);
                const float fd2 = fx * fx + fy * fy + fz * fz;
                const float4 v0 = __ldg(A.thin + node);
                const float4 v1 = __ldg(A.thick + node);
                const float rx = fx + v0.z, ry = fy + v0.w, rz = fz + v1.x;
                // mapping at the centre of luminosity (Sec. 7.6): segment, straddles and key
                // at the COL position for nodes whose COL is off centre (col_decide)
                const bool colmap = GENERAL && A.col_mapping && (v0.z != 0.0f || v0.w != 0.0f || v1.x != 0.0f);
                const int elog = A.lmax - lvl + 1;
                int i, Kx, Ky, Kz, cilo = 0, cihi = 0;
                if (colmap) {
                    const ColMap cm = col_decide(A, node, ox, oy, oz, rx, ry, rz, lvl, tl, lp, THICK && v1.w > 0.0f);
                    i = cm.i;
                    Kx = cm.kx;
                    Ky = cm.ky;
                    Kz = cm.kz;
                    cilo = cm.ilo;
                    cihi = cm.ihi;
                } else {
                    i = fixup_pair(guess_bin(fd2, lp), d2, thr2, nb);
                    Kx = alpha_key(ox, elog);
                    Ky = alpha_key(oy, elog);
                    Kz = alpha_key(oz, elog);
                }
                // one approximate reciprocal per node (MUFU, ~1 ulp) serves beta and the depth
                const float inv_r2 = __fdividef(1.0f, rx * rx + ry * ry + rz * rz);
                const float beta = __ldg(R2 + i) * inv_r2;
                if (abs(Kx) > A.D || abs(Ky) > A.D || abs(Kz) > A.D) {
                    atomicOr(A.err, kErrAlphaKey);
                } else {
                    const int idx = ((Kz + A.D) * W + (Ky + A.D)) * W + (Kx + A.D);
                    const int2 ee = __ldg(s_apair + idx);
                    const int e0 = ee.x, e1 = ee.y;
                    if (e1 == e0) atomicOr(A.err, kErrAlphaKey);
                    // a node without thin material (all of it thick) adds nothing to the thin
                    // tile: its entries are left out of the warp's thin deposits
                    ne = (!THICK || v0.x != 0.0f || v0.y != 0.0f) ? e1 - e0 : 0;
                    ebase = e0;
                    cbase = i * ROW;
                    bL = beta * v0.x * A.inv_s3;
                    bA = beta * v0.y * A.inv_s3;
                    if (THICK && v1.w > 0.0f) {
                        int ilo = cilo, ihi = cihi;
                        if (!colmap) {
                            const int64_t* lo = A.str_lo + ((int64_t)tl * (A.lmax + 1) + lvl) * nb;
                            const int64_t* hi = A.str_hi + ((int64_t)tl * (A.lmax + 1) + lvl) * nb;
                            const float d = sqrtf(fd2);
                            const float sd = 0.8660254f * (float)(2 << (A.lmax - lvl));
                            const float dl = fmaxf(d - sd, 0.0f), dh = d + sd;
                            ilo = fixup(guess_bin(dl * dl, lp), d2, lo, nb);
                            ihi = fixup(guess_bin(dh * dh, lp), d2, hi, nb);
                        }
                        unsigned long long fmask = 0ull;
                        for (int j = ilo; j < ihi; ++j) fmask |= 1ull << j;
                        nk = e1 - e0;
                        kLV = v1.y;
                        kA = v1.z;
                        kV = v1.w;
                        kbeta = beta;
                        kfm = fmask;
                    }
                }
            }
            // warp-level exclusive scan of the entry counts,
            // in child-major order (child c of the warp's groups 0..3, then child c + 1, ...):
            // entries of sibling nodes, which often share a cell, fall into different rounds
            const int nv = __shfl_sync(full, ne, ((lane & 3) << 3) | (lane >> 2));
            int inc = nv;
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(full, inc, off);
                if (lane >= off) inc += t;
            }
            const int tw = __shfl_sync(full, inc, 31);
            const int pre = __shfl_sync(full, inc - nv, ((lane & 7) << 2) | (lane >> 3));
            if (tw > 0) {
                if (tw <= OCAP) {
                    if (ne > 0) {
                        for (int k = 0; k < ne; ++k) owner[pre + k] = (unsigned char)lane;
                    }
                    __syncwarp();
                    // two entries per lane per pass; each entry's node data comes from its
                    // owner lane by shuffles (warp-uniform passes, full-mask shuffles)
                    const int eb = ebase - pre;
                    for (int r0 = 0; r0 < tw; r0 += 64) {
                        const int r = r0 + lane, r2 = r + 32;
                        const int o1 = r < tw ? (int)owner[r] : 0;
                        const int o2 = r2 < tw ? (int)owner[r2] : 0;
                        const int4 nd = make_int4(__shfl_sync(full, cbase, o1), __shfl_sync(full, eb, o1),
                                                  __shfl_sync(full, __float_as_int(bL), o1),
                                                  __shfl_sync(full, __float_as_int(bA), o1));
                        const int4 nd2 = make_int4(__shfl_sync(full, cbase, o2), __shfl_sync(full, eb, o2),
                                                   __shfl_sync(full, __float_as_int(bL), o2),
                                                   __shfl_sync(full, __float_as_int(bA), o2));
                        const uint32_t ent = r < tw ? __ldg(A.aent + nd.y + r) : 0u;
                        const uint32_t ent2 = r2 < tw ? __ldg(A.aent + nd2.y + r2) : 0u;
                        if (r < tw) {
                            const int c = nd.x + (int)(ent & 0xffffu);
                            const float w = count_to_float(ent >> 16);
                            deposit_thin(tL, c, w * __int_as_float(nd.z), w * __int_as_float(nd.w));
                        }
                        if (r2 < tw) {
                            const int c2 = nd2.x + (int)(ent2 & 0xffffu);
                            const float w2 = count_to_float(ent2 >> 16);
                            deposit_thin(tL, c2, w2 * __int_as_float(nd2.z), w2 * __int_as_float(nd2.w));
                        }
                    }
                    __syncwarp();
                } else {
                    for (int e = ebase; e < ebase + ne; ++e) {
                        const uint32_t ent = __ldg(A.aent + e);
                        const int c = cbase + (int)(ent & 0xffffu);
                        const float w = count_to_float(ent >> 16);
                        deposit_thin(tL, c, w * bL, w * bA);
                    }
                }
            }
            if constexpr (THICK) {
                // thick deposits: one entry per lane per pass, the node data from the owner
                // lane by shuffles; owners recorded in the same per-warp byte array, which
                // the thin passes above have finished reading
                if (__any_sync(full, nk > 0)) {
                    int tinc = nk;
                    for (int off = 1; off < 32; off <<= 1) {
                        const int t = __shfl_up_sync(full, tinc, off);
                        if (lane >= off) tinc += t;
                    }
                    const int tt = __shfl_sync(full, tinc, 31);
                    const int tpre = tinc - nk;
                    if (tt <= OCAP) {
                        __syncwarp();
                        for (int k = 0; k < nk; ++k) owner[tpre + k] = (unsigned char)lane;
                        __syncwarp();
                        const int teb = ebase - tpre;
                        for (int r0 = 0; r0 < tt; r0 += 32) {
                            const int r = r0 + lane;
                            const int o = r < tt ? (int)owner[r] : 0;
                            const int cb = __shfl_sync(full, cbase, o), eb = __shfl_sync(full, teb, o);
                            const float y = __shfl_sync(full, kLV, o), z = __shfl_sync(full, kA, o);
                            const float v = __shfl_sync(full, kV, o), bt = __shfl_sync(full, kbeta, o);
                            const unsigned long long fm = __shfl_sync(full, kfm, o);
                            if (r < tt) {
                                const uint32_t ent = __ldg(A.aent + eb + r);
                                const int h = (int)(ent & 0xffffu);
                                const int cidx = cb + h;
                                const float wn = count_to_float(ent >> 16) * A.inv_s3;
                                atomicAdd(tLk + cidx, wn * y);
                                atomicAdd(tAk + cidx, z);
                                atomicAdd(tVk + cidx, wn * v);
                                atomicAdd(tQk + cidx, wn * bt * v);
                                if (fm) atomicOr(flags + h, fm);
                            }
                        }
                        __syncwarp();
                    } else {
                        for (int e = ebase; e < ebase + nk; ++e) {
                            const uint32_t ent = __ldg(A.aent + e);
                            const int h = (int)(ent & 0xffffu);
                            const int cidx = cbase + h;
                            const float wn = count_to_float(ent >> 16) * A.inv_s3;
                            atomicAdd(tLk + cidx, wn * kLV);
                            atomicAdd(tAk + cidx, kA);
                            atomicAdd(tVk + cidx, wn * kV);
                            atomicAdd(tQk + cidx, wn * kbeta * kV);
                            if (kfm) atomicOr(flags + h, kfm);
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (s_overflow) {
            if (tid == 0) atomicOr(A.err, kErrStack);
            __syncthreads();
            continue;
        }
        // ---- own cell: segment 0 of every ray, alpha = 1/N_pix, beta = 1
        {
            const float4 v0 = __ldg(A.thin + tnode);
            const float4 v1 = __ldg(A.thick + tnode);
            unsigned long long fmask = 0ull;
            if (THICK && v1.w > 0.0f) {
                const int64_t* hi = A.str_hi + ((int64_t)tl * (A.lmax + 1) + tl) * nb;
                int ihi = 0;
                for (int j = 1; j < nb; ++j) ihi += 0 >= __ldg(hi + j);
                for (int j = 0; j < ihi; ++j) fmask |= 1ull << j;
            }
            const float w = 1.0f / NPIX;
            for (int h = tid; h < NPIX; h += NT) {
                gst(tL + LS * h, gld(tL + LS * h) + w * v0.x);
                gst(tA + LS * h, gld(tA + LS * h) + w * v0.y);
                if (THICK && v1.w > 0.0f) {
                    gst(tLk + h, gld(tLk + h) + w * v1.y);
                    gst(tAk + h, gld(tAk + h) + v1.z);
                    gst(tVk + h, gld(tVk + h) + w * v1.w);
                    gst(tQk + h, gld(tQk + h) + w * v1.w);
                    gst64(flags + h, gld64(flags + h) | fmask);
                }
            }
        }
        __syncthreads();
        // eq. merge (Sec. 4.3): a flagged boundary between segments i and i+1 lies inside a thick
        // node, so segment i+1 folds into i (thin content and Q^_thick scaled by R_i^2/R_(i+1)^2,
        // the other thick sums added), from the outside in; one thread per ray
        auto merge_flagged = [&](int h) {
            const unsigned long long fl = gld64(flags + h);
            if (fl)
                for (int i = nb - 2; i >= 0; --i) {
                    if (!((fl >> i) & 1ull)) continue;
                    const int c0 = i * ROW + h, c1 = (i + 1) * ROW + h;
                    const float T = __ldg(R2 + i) / __ldg(R2 + i + 1);
                    gst(tL + LS * c0, gld(tL + LS * c0) + T * gld(tL + LS * c1));
                    gst(tA + LS * c0, gld(tA + LS * c0) + T * gld(tA + LS * c1));
                    gst(tQk + c0, gld(tQk + c0) + T * gld(tQk + c1));
                    gst(tLk + c0, gld(tLk + c0) + gld(tLk + c1));
                    gst(tAk + c0, gld(tAk + c0) + gld(tAk + c1));
                    gst(tVk + c0, gld(tVk + c0) + gld(tVk + c1));
                    gst(tL + LS * c1, 0.0f);
                    gst(tA + LS * c1, 0.0f);
                    for (float* q : {tQk, tLk, tAk, tVk}) gst(q + c1, 0.0f);
                }
        };
        // ---- integrate each ray from the inside out
        // J sums positive FP32 terms. The flux vector cancels between opposite rays, so each
        // product F^h n^h is split exactly into a float pair and summed with error-free
        // transformations. No FP64 on the way.
        //
        // Segments i0 <= i < i1 of ray h, attenuated only by the segments of the range inside them:
        //   Fp = sum_i eps_i F*_i,  et = prod_i e^-tau_thin,i,  ek = prod_i thick transmission,
        //   ts = sum_i tau_thin,i.
        auto segments = [&](int h, int i0, int i1, float& Fp, float& et, float& ek, float& ts) {
            for (int i = i0; i < i1; ++i) {
                const int ci = i * ROW + h;
                const float Lth = gld(tL + LS * ci);
                const float R2i = __ldg(R2 + i);
                const float inv_R2 = __fdividef(1.0f, R2i);
                const float Ath = gld(tA + LS * ci);
                const float tth = i == 0 ? 0.0f : Ath * inv_R2 * (1.0f / omega);  // eq. tauthin
                const float Vk = THICK ? gld(tVk + ci) : 0.0f;
                if (Lth == 0.0f && Ath == 0.0f && Vk == 0.0f) continue;  // empty segment
                float f = 0.0f, Fk = 0.0f, Akv = 0.0f, tk = 0.0f;
                if constexpr (THICK) {
                    if (Vk > 0.0f) {
                        const float cb = cbrtf(Vk);
                        float wk = (gld(tQk + ci) / Vk) * (cb * cb) * inv_R2;
                        wk = fminf(wk, omega);
                        f = wk / omega;
                        Akv = gld(tAk + ci);
                        tk = (i == 0 || wk == 0.0f) ? 0.0f : Akv / (wk * R2i);
                        Fk = wk * gld(tLk + ci) / Vk;
                    }
                }
                // g = (1 - e^-tau) / tau (eq. fthin, the escape fraction of the segment's own
                // emission) and its transmission e^-tau = 1 - tau g: a series below 1/16
                // (truncation below 2e-9), exp above
                float g, eth;
                if (tth < 0.0625f) {
                    g = fmaf(tth, fmaf(tth, fmaf(tth, fmaf(tth, 1.0f / 120.0f, -1.0f / 24.0f), 1.0f / 6.0f), -0.5f),
                             1.0f);
                    eth = fmaf(-tth, g, 1.0f);
                } else {
                    eth = expf(-tth);
                    g = (1.0f - eth) * __fdividef(1.0f, tth);
                }
                const float Fth = g * Lth * inv_R2 * (float)(1.0 / (4.0 * kPi));
                // eq. fcombined; without thick material the blend is F*_thin itself
                float Fs = Fth;
                if constexpr (THICK) {
                    const float den = Ath + f * Akv;
                    Fs = den > 0.0f ? (Fth * Ath + Fk * f * Akv) / den : Fth + Fk;
                }
                // eq. ext inner: the segments inside attenuate by the product of their thin
                // transmissions (each e^-tau to FP32 rounding, so the product keeps its relative
                // precision at any depth) and of their thick ones
                Fp += et * ek * Fs;
                ts += tth;
                et *= eth;
                if (THICK && f > 0.0f) ek *= (1.0f - f) + f * expf(-tk);
            }
        };
        float Js = 0.0f;
        float Fxh = 0.0f, Fxl = 0.0f, Fyh = 0.0f, Fyl = 0.0f, Fzh = 0.0f, Fzl = 0.0f;
        float tsum = 0.0f, tminv = 3.0e38f;
        auto ray_done = [&](int h, float Fh, float tr) {
            if (A.tau_mean) {
                tsum += tr;
                tminv = fminf(tminv, tr);
            }
            Js += Fh;
            const float* nh = s_nhat;
            add_product(Fxh, Fxl, -Fh, __ldg(nh + 3 * h));
            add_product(Fyh, Fyl, -Fh, __ldg(nh + 3 * h + 1));
            add_product(Fzh, Fzl, -Fh, __ldg(nh + 3 * h + 2));
        };
        // tiles with spare threads: the segments of a ray are cut into P consecutive parts, one
        // thread each; a part's result is carried outward by the transmission of the parts
        // inside it
        constexpr int P = NT >= 4 * NPIX ? 4 : (NT >= 2 * NPIX ? 2 : 1);
        if constexpr (THICK && P > 1) {
            // thick tiles split too: the merges of straddled boundaries first (Sec. 4.3), one
            // thread per ray; a part then hands on its total transmission, thin times thick
            if (nb >= 2 * P) {
                for (int h = tid; h < NPIX; h += NT) merge_flagged(h);
                __syncthreads();
            }
        }
        if (P > 1 && nb >= 2 * P) {
            if (tid < P * NPIX) {
                const int h = tid % NPIX, p = tid / NPIX;
                const int i0 = p * nb / P, i1 = (p + 1) * nb / P;
                float Fp = 0.0f, et = 1.0f, ek = 1.0f, ts = 0.0f;
                segments(h, i0, i1, Fp, et, ek, ts);
                // every part has >= 2 segments: its first two cells of ray h, read only by
                // this thread, now hold (Fp, transmission) and the part's optical depth
                gst(tL + LS * (i0 * ROW + h), Fp);
                gst(tA + LS * (i0 * ROW + h), et * ek);
                gst(tL + LS * ((i0 + 1) * ROW + h), ts + (THICK && ek < 1.0f ? -__logf(ek) : 0.0f));
            }
            __syncthreads();
            if (tid < NPIX) {
                const int h = tid;
                float Fh = 0.0f, tr = 1.0f, ts = 0.0f;
                for (int p = 0; p < P; ++p) {
                    const int i0 = p * nb / P;
                    Fh += tr * gld(tL + LS * (i0 * ROW + h));
                    tr *= gld(tA + LS * (i0 * ROW + h));
                    ts += gld(tL + LS * ((i0 + 1) * ROW + h));
                }
                ray_done(h, Fh, ts);
            }
        } else {
            for (int h = tid; h < NPIX; h += NT) {
                if (THICK) merge_flagged(h);
                float Fh = 0.0f, et = 1.0f, ek = 1.0f, ts = 0.0f;
                segments(h, 0, nb, Fh, et, ek, ts);
                // optical depth of the whole ray: thin depths plus thick transmission
                ray_done(h, Fh, ts + (THICK && ek < 1.0f ? -__logf(ek) : 0.0f));
            }
        }
        // ---- team reduction (only warps that hold rays contribute)
        if (warp * 32 < NPIX) {
            for (int off = 16; off > 0; off >>= 1) {
                Js += __shfl_xor_sync(full, Js, off);
                const float xh = __shfl_xor_sync(full, Fxh, off), xl = __shfl_xor_sync(full, Fxl, off);
                const float yh = __shfl_xor_sync(full, Fyh, off), yl = __shfl_xor_sync(full, Fyl, off);
                const float zh = __shfl_xor_sync(full, Fzh, off), zl = __shfl_xor_sync(full, Fzl, off);
                add_pair(Fxh, Fxl, xh, xl);
                add_pair(Fyh, Fyl, yh, yl);
                add_pair(Fzh, Fzl, zh, zl);
            }
            if (lane == 0) {
                s_red[0][warp] = Js;
                s_red[1][warp] = Fxh;
                s_red[2][warp] = Fxl;
                s_red[3][warp] = Fyh;
                s_red[4][warp] = Fyl;
                s_red[5][warp] = Fzh;
                s_red[6][warp] = Fzl;
            }
            if (A.tau_mean) {
                for (int off = 16; off > 0; off >>= 1) {
                    tsum += __shfl_xor_sync(full, tsum, off);
                    tminv = fminf(tminv, __shfl_xor_sync(full, tminv, off));
                }
                if (lane == 0) {
                    s_tau[0][warp] = tsum;
                    s_tau[1][warp] = tminv;
                }
            }
        }
        __syncthreads();
        // four lanes of warp 0 write J and the three flux components in CGS
        if (tid < 4) {
            const double Fu = A.scal[0] * A.inv_u2;  // internal flux unit in erg/s/cm^2
            if (tid == 0) {
                float js = 0.0f;
                for (int w = 0; w < WPT && w * 32 < NPIX; ++w) js += s_red[0][w];
                const int64_t k = A.perm[s];
                A.J[out] = (float)((double)js * (Fu * (1.0 / (4.0 * kPi))) + A.jsrc[k]);
            } else {
                float hi = 0.0f, lo = 0.0f;
                for (int w = 0; w < WPT && w * 32 < NPIX; ++w) add_pair(hi, lo, s_red[2 * tid - 1][w], s_red[2 * tid][w]);
                A.F[3 * out + tid - 1] = ((double)hi + (double)lo) * Fu;
            }
            if (tid == 0 && A.tau_mean) {
                float ts = 0.0f, tm = 3.0e38f;
                for (int w = 0; w < WPT && w * 32 < NPIX; ++w) {
                    ts += s_tau[0][w];
                    tm = fminf(tm, s_tau[1][w]);
                }
                A.tau_mean[out] = ts / NPIX;
                A.tau_min[out] = tm;
            }
        }
        __syncthreads();
    }
}

template <int NPIX, bool THICK, int WPT, bool GENERAL>
__global__ void __launch_bounds__(WPT * 32, min_warps_per_sm(NPIX, THICK) / WPT)
    k_evaluate(const __grid_constant__ EvalArgs a) {
    evaluate_team<NPIX, THICK, WPT, GENERAL, false>(a, nullptr);
}

// batches run teams of 2 or 3 (thin tiles) or 4 warps
template <int NPIX, bool THICK, int WPT, bool GENERAL>
__global__ void __launch_bounds__(WPT * 32, min_warps_per_sm(NPIX, THICK) / WPT)
    k_evaluate_batch(const __grid_constant__ BatchArgs p) {
    evaluate_team<NPIX, THICK, WPT, GENERAL, true>(p.launch, &p);
}

template <typename K>
treeray_status launch_persistent(treeray_ctx* c, K kern, size_t per_warp, int max_warps, int64_t n,
                                 unsigned long long* queue, cudaStream_t s, const EvalArgs& a) {
    int smem_optin = 0, sms = 0;
    TR_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    int warps = max_warps;
    while (warps > 1 && per_warp * warps > (size_t)smem_optin) --warps;
    if (per_warp * warps > (size_t)smem_optin) {
        set_error("evaluate: a warp's walk scratch exceeds shared memory");
        return TREERAY_EINVAL;
    }
    const size_t smem = per_warp * warps;
    TR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
    if (per_sm < 1) {
        set_error("evaluate: kernel does not fit on an SM");
        return TREERAY_EINVAL;
    }
    int64_t blocks = (int64_t)per_sm * sms;
    const int64_t need = (n + warps - 1) / warps;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    TR_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s));
    kern<<<(int)blocks, warps * 32, smem, s>>>(a);
    c->launches += 1;
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}

// Global-memory tiles of one launch are kept within this many bytes. Tiles beyond the 129 MB
// L2 go through HBM, which costs less than teams left unlaunched: 768 rays on the collapsing
// core (thick tiles of 369 KB) took 5577 ms with one launch's tiles capped at 96 MB and 2525
// ms at 1 GB (192 rays: 436 -> 408 ms).
constexpr size_t kGlobalTileBudget = (size_t)1 << 30;

// Bytes of one team's slice of global memory (the tile, then the thick merge flags),
// 16-byte aligned.
size_t team_tile_bytes(int npix, int nbins, bool thick) {
    const int nq = thick ? 6 : 2;
    return align16(align16((size_t)nq * nbins * tile_row(npix, thick) * 4) + (thick ? (size_t)npix * 8 : 0));
}

// Teams of a launch: those asked for, at most as many as keep their tiles within the L2
// budget (but one per SM).
int64_t tile_blocks(size_t tile_bytes, int64_t want, int sms) {
    return std::max<int64_t>(1, std::min<int64_t>(want, std::max<int64_t>(sms, (int64_t)(kGlobalTileBudget / tile_bytes))));
}

treeray_status reserve_global_tiles(treeray_ctx* c, size_t bytes, cudaStream_t s) {
    if (c->gtile_bytes >= bytes) return TREERAY_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    TR_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        set_error("evaluate: team tiles must be reserved before stream capture (build or evaluate first)");
        return TREERAY_EINVAL;
    }
    if (c->gtile) {
        TR_CUDA(cudaFree(c->gtile));  // waits for launches that may still use it
        c->gtile = nullptr;
        c->gtile_bytes = 0;
    }
    const treeray_status rc = dev_alloc(c, (void**)&c->gtile, bytes);
    if (rc != TREERAY_OK) return rc;
    c->gtile_bytes = bytes;
    return TREERAY_OK;
}

size_t stack_bytes_for(int wpt, int lmax, int blocks) {
    // the team stack holds at most one batch of pushes (32 WPT groups) per level
    return (size_t)blocks * (size_t)(32 * wpt * (lmax + 1) + 64) * sizeof(int);
}

template <int NPIX, bool THICK, int WPT, bool GENERAL, bool BATCH>
treeray_status launch_team(treeray_ctx* c, const EvalArgs& a, const EvalArgs* boxes,
                           const int64_t* box_start, int nbox, int layout_lmax, cudaStream_t s) {
    // batch: boxes and box_start are HOST arrays of the boxes' descriptors and first targets
    EvalArgs b = a;
    b.stack_cap = (int)(stack_bytes_for(WPT, layout_lmax, 1) / sizeof(int));
    if (c->stack_limit > 0) b.stack_cap = std::min(b.stack_cap, c->stack_limit);  // test hook
    const size_t tile_bytes = team_tile_bytes(NPIX, a.nbins, THICK);
    const size_t smem = (size_t)WPT * owner_cap_for(NPIX, THICK);
    int smem_optin = 0, sms = 0;
    TR_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    if (smem + 2048 > (size_t)smem_optin) {
        set_error("evaluate: a team's owner bytes exceed shared memory");
        return TREERAY_EINVAL;
    }
    // persistent grid for n targets: resident blocks of the kernel, and team stacks for them
    auto grid_for = [&](auto kern, int64_t n, int64_t& blocks) -> treeray_status {
        TR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        TR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPT * 32, smem));
        if (per_sm < 1) {
            set_error("evaluate: kernel does not fit on an SM");
            return TREERAY_EINVAL;
        }
        // the autotuner may launch fewer resident teams than fit (occ_pct of them, >= 1 per SM)
        const int use = std::max(1, (per_sm * c->occ_pct + 50) / 100);
        blocks = tile_blocks(tile_bytes, std::min<int64_t>((int64_t)use * sms, n), sms);
        const treeray_status rg = reserve_global_tiles(c, (size_t)blocks * tile_bytes, s);
        if (rg != TREERAY_OK) return rg;
        if (c->stack_scr_bytes < stack_bytes_for(WPT, layout_lmax, (int)blocks)) {
            const treeray_status rc = reserve_eval_stacks(c, layout_lmax, s);
            if (rc != TREERAY_OK) return rc;
        }
        return TREERAY_OK;
    };
    int64_t blocks = 0;
    treeray_status rc;
    if constexpr (!BATCH) {
        auto kern = k_evaluate<NPIX, THICK, WPT, GENERAL>;
        if ((rc = grid_for(kern, a.n, blocks)) != TREERAY_OK) return rc;
        b.stack = c->stack_scr;
        b.gtile = c->gtile;
        b.gtile_stride = (int64_t)(tile_bytes / sizeof(float));
        TR_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s));
        kern<<<(int)blocks, WPT * 32, smem, s>>>(b);
        c->launches += 1;
        TR_CUDA(cudaGetLastError());
    } else {
        static_assert(WPT == 4 || ((WPT == 2 || WPT == 3) && !THICK), "batches run teams of 2, 3 (thin) or 4 warps");
        auto kern = k_evaluate_batch<NPIX, THICK, WPT, GENERAL>;
        std::unique_ptr<BatchArgs> p(new (std::nothrow) BatchArgs());
        if (!p) {
            set_error("out of host memory");
            return TREERAY_ENOMEM;
        }
        for (int c0 = 0; c0 < nbox; c0 += kMaxLaunchBoxes) {  // one launch per chunk of boxes
            const int c1 = std::min(nbox, c0 + kMaxLaunchBoxes);
            p->launch = b;
            p->launch.n = box_start[c1] - box_start[c0];
            p->nbox = c1 - c0;
            for (int k = 0; k < c1 - c0; ++k) {
                p->box[k] = boxes[c0 + k];
                p->start[k] = box_start[c0 + k] - box_start[c0];
            }
            p->start[c1 - c0] = p->launch.n;
            if (p->launch.n == 0) continue;
            if ((rc = grid_for(kern, p->launch.n, blocks)) != TREERAY_OK) return rc;
            p->launch.stack = c->stack_scr;
            p->launch.gtile = c->gtile;
            p->launch.gtile_stride = (int64_t)(tile_bytes / sizeof(float));
            TR_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s));
            kern<<<(int)blocks, WPT * 32, smem, s>>>(*p);
            c->launches += 1;
            TR_CUDA(cudaGetLastError());
        }
    }
    return TREERAY_OK;
}

template <int NPIX, bool THICK, bool GENERAL>
treeray_status launch_wpt(treeray_ctx* c, int wpt, const EvalArgs& a, const EvalArgs* boxes,
                          const int64_t* box_start, int nbox, int layout_lmax, cudaStream_t s) {
    if constexpr (WideRays<NPIX>::on) {  // 768 rays: teams of 2, 4 or 8 warps, no batches
        if (boxes) {
            set_error("batch: 768 rays are evaluated one box at a time");
            return TREERAY_EINVAL;
        }
        if (wpt == 2) return launch_team<NPIX, THICK, 2, GENERAL, false>(c, a, nullptr, nullptr, 0, layout_lmax, s);
        if (wpt == 8) return launch_team<NPIX, THICK, 8, GENERAL, false>(c, a, nullptr, nullptr, 0, layout_lmax, s);
        return launch_team<NPIX, THICK, 4, GENERAL, false>(c, a, nullptr, nullptr, 0, layout_lmax, s);
    } else {
    // batches run teams of 2 or 3 warps (thin tiles, when that is the team size asked for) or 4
    if (boxes) {
        if constexpr (!THICK) {
            if (wpt == 2) return launch_team<NPIX, THICK, 2, GENERAL, true>(c, a, boxes, box_start, nbox, layout_lmax, s);
            if (wpt == 3) return launch_team<NPIX, THICK, 3, GENERAL, true>(c, a, boxes, box_start, nbox, layout_lmax, s);
        }
        return launch_team<NPIX, THICK, 4, GENERAL, true>(c, a, boxes, box_start, nbox, layout_lmax, s);
    }
    switch (wpt) {
        case 2: return launch_team<NPIX, THICK, 2, GENERAL, false>(c, a, nullptr, nullptr, 0, layout_lmax, s);
        case 3:  // thin tiles only; thick teams of three were slower than four
            if constexpr (!THICK) return launch_team<NPIX, THICK, 3, GENERAL, false>(c, a, nullptr, nullptr, 0, layout_lmax, s);
            return launch_team<NPIX, THICK, 4, GENERAL, false>(c, a, nullptr, nullptr, 0, layout_lmax, s);
        case 8: return launch_team<NPIX, THICK, 8, GENERAL, false>(c, a, nullptr, nullptr, 0, layout_lmax, s);
        default: return launch_team<NPIX, THICK, 4, GENERAL, false>(c, a, nullptr, nullptr, 0, layout_lmax, s);
    }
    }
}

template <int NPIX>
treeray_status launch_kind(treeray_ctx* c, bool thick, bool periodic, int wpt, const EvalArgs& a,
                           const EvalArgs* boxes, const int64_t* box_start, int nbox, int layout_lmax,
                           cudaStream_t s) {
    // the general instantiations carry the closest-copy and COL-mapping code; isolated grids
    // mapped at geometric centres run without it
    if (periodic)
        return thick ? launch_wpt<NPIX, true, true>(c, wpt, a, boxes, box_start, nbox, layout_lmax, s)
                     : launch_wpt<NPIX, false, true>(c, wpt, a, boxes, box_start, nbox, layout_lmax, s);
    return thick ? launch_wpt<NPIX, true, false>(c, wpt, a, boxes, box_start, nbox, layout_lmax, s)
                 : launch_wpt<NPIX, false, false>(c, wpt, a, boxes, box_start, nbox, layout_lmax, s);
}

treeray_status dispatch_team(treeray_ctx* c, bool thick, bool periodic, int wpt, const EvalArgs& a,
                             const EvalArgs* boxes, const int64_t* box_start, int nbox, int layout_lmax,
                             cudaStream_t s) {
    switch (c->p.npix) {
        case 12: return launch_kind<12>(c, thick, periodic, wpt, a, boxes, box_start, nbox, layout_lmax, s);
        case 48: return launch_kind<48>(c, thick, periodic, wpt, a, boxes, box_start, nbox, layout_lmax, s);
        case 192: return launch_kind<192>(c, thick, periodic, wpt, a, boxes, box_start, nbox, layout_lmax, s);
        case 768: return launch_kind<768>(c, thick, periodic, wpt, a, boxes, box_start, nbox, layout_lmax, s);
    }
    set_error("evaluate: npix must be 12, 48, 192 or 768");
    return TREERAY_EINVAL;
}

// The general kernels carry periodic closest copies and mapping at the COL; the others map
// isolated grids at the geometric centres.
bool needs_general(const treeray_ctx* c) { return c->p.periodic != 0 || c->p.col_mapping != 0; }

treeray_status dispatch_eval(treeray_ctx* c, const EvalArgs& a, cudaStream_t s) {
    return dispatch_team(c, c->has_thick || c->force_thick, needs_general(c), c->wpt, a, nullptr, nullptr, 1,
                         c->lmax, s);
}

treeray_status dispatch_list(treeray_ctx* c, const EvalArgs& a, cudaStream_t s) {
    return launch_persistent(c, k_walk_list, (size_t)a.stack_cap * 4, 8, a.n, a.queue, s, a);
}

EvalArgs make_args(treeray_ctx* c, const int32_t* targets, int64_t n) {
    EvalArgs a{};
    a.geo = c->tree.geo;
    a.thin = c->tree.thin;
    a.thick = c->tree.thick;
    a.leaf_node = c->tree.leaf_node;
    a.perm = c->tree.perm;
    a.inv_perm = c->tree.inv_perm;
    a.targets = targets;
    a.jsrc = c->tree.jsrc;
    a.nhat = c->dt.nhat;
    a.aoff = c->dt.alpha_off;
    a.apair = c->dt.alpha_pair;
    a.aent = c->dt.alpha_ent;
    a.orient = c->rot.empty() ? nullptr : c->orient;
    a.aoff_stride = (int64_t)(2 * c->ht.D + 1) * (2 * c->ht.D + 1) * (2 * c->ht.D + 1) + 1;
    a.bin_thr = c->dt.bin_thr;
    a.bin_thr2 = c->dt.bin_thr2;
    a.R2 = c->dt.R2;
    a.Rh = c->dt.Rh;
    a.Rd = c->dt.Rd;
    a.mom = c->tree.mom;
    a.nn = c->nnodes;
    a.open_max = c->dt.open_max;
    a.str_lo = c->dt.str_lo;
    a.str_hi = c->dt.str_hi;
    a.lvlp = c->dt.lvlp;
    a.scal = c->dt.scal;
    a.err = c->dt.err;
    a.queue = c->dt.queue;
    a.n = n;
    a.nleaves = c->nleaves;
    a.lmax = c->lmax;
    a.nbins = c->p.nbins;
    a.D = c->ht.D;
    a.npix = c->p.npix;
    a.periodic = c->p.periodic;
    a.col_mapping = c->p.col_mapping;
    a.inv_s3 = 1.0f / (float)(c->ht.s * c->ht.s * c->ht.s);
    a.u = c->u;
    a.inv_u2 = 1.0 / (c->u * c->u);
    // the stack holds at most 28 leftover groups per level plus one batch of pushes
    a.stack_cap = 28 * (c->lmax + 1) + 40;
    if (c->stack_limit > 0) a.stack_cap = std::min(a.stack_cap, c->stack_limit);  // test hook
    return a;
}

}  // namespace

treeray_status reserve_eval_stacks(treeray_ctx* c, int lmax, cudaStream_t s) {
    int sms = 0;
    TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    // at most 2048 threads, i.e. 64 / WPT teams, per SM
    size_t need = 0;
    for (int wpt : {2, 3, 4, 8}) need = std::max(need, stack_bytes_for(wpt, lmax, sms * (64 / wpt)));
    if (c->stack_scr_bytes >= need) return TREERAY_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    TR_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        set_error("evaluate: team-stack scratch must be reserved before stream capture (build first)");
        return TREERAY_EINVAL;
    }
    if (c->stack_scr) {
        TR_CUDA(cudaFree(c->stack_scr));  // waits for launches that may still use it
        c->stack_scr = nullptr;
        c->stack_scr_bytes = 0;
    }
    const treeray_status rc = dev_alloc(c, (void**)&c->stack_scr, need);
    if (rc != TREERAY_OK) {
        c->stack_scr = nullptr;
        return rc;
    }
    c->stack_scr_bytes = need;
    return TREERAY_OK;
}

// The teams' tiles for up to n targets, for each kind of tile (thin or thick) a launch of
// this context can use and any team size, so that launches captured in a CUDA graph find
// them reserved.
treeray_status reserve_team_tiles_kind(treeray_ctx* c, int64_t n, bool thick, cudaStream_t s) {
    int sms = 0;
    TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const size_t tb = team_tile_bytes(c->p.npix, c->p.nbins, thick);
    // at most 2048 threads, i.e. 32 teams of 2 warps, per SM
    const int64_t teams = tile_blocks(tb, std::min<int64_t>(std::max<int64_t>(n, 1), 32LL * sms), sms);
    return reserve_global_tiles(c, tb * (size_t)teams, s);
}

treeray_status reserve_team_tiles(treeray_ctx* c, int64_t n, cudaStream_t s) {
    // thick tiles for trees with thick material, thin tiles for trees without; both where a
    // refresh can change the classes (temperature-dependent opacity)
    for (bool thick : {false, true}) {
        const bool tdep = c->p.kappa_model == 1;
        const bool possible = thick ? (c->has_thick || c->force_thick || tdep) : (!c->has_thick || tdep);
        if (!possible) continue;
        const treeray_status rc = reserve_team_tiles_kind(c, n, thick, s);
        if (rc != TREERAY_OK) return rc;
    }
    return TREERAY_OK;
}

treeray_status launch_evaluate(treeray_ctx* c, const int32_t* targets, int64_t n, float* J, double* F,
                               cudaStream_t s) {
    EvalArgs a = make_args(c, targets, n);
    a.J = J;
    a.F = F;
    return dispatch_eval(c, a, s);
}

treeray_status launch_evaluate_tau(treeray_ctx* c, float* J, double* F, float* tau_mean, float* tau_min,
                                   cudaStream_t s) {
    EvalArgs a = make_args(c, nullptr, c->nleaves);
    a.J = J;
    a.F = F;
    a.tau_mean = tau_mean;
    a.tau_min = tau_min;
    return dispatch_eval(c, a, s);
}

treeray_status launch_evaluate_skip(treeray_ctx* c, float* J, double* F, const int* skip, cudaStream_t s) {
    EvalArgs a = make_args(c, nullptr, c->nleaves);
    a.J = J;
    a.F = F;
    a.skip = skip;
    return dispatch_eval(c, a, s);
}

treeray_status launch_accepted(treeray_ctx* c, const int32_t* targets, int64_t n, int32_t cap,
                               int32_t* counts, int32_t* ids, cudaStream_t s) {
    EvalArgs a = make_args(c, targets, n);
    a.acc_counts = counts;
    a.acc_ids = ids;
    a.acc_cap = cap;
    return dispatch_list(c, a, s);
}

treeray_status launch_walk_stats(treeray_ctx* c, const int32_t* targets, int64_t n, int64_t* totals,
                                 cudaStream_t s) {
    EvalArgs a = make_args(c, targets, n);
    a.stats = reinterpret_cast<unsigned long long*>(totals);
    a.acc_cap = 0;
    return dispatch_list(c, a, s);
}


namespace {
__global__ void k_sample_targets(int32_t* t, int64_t n, int64_t N, int64_t step) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) t[i] = (int32_t)((i * step) % N);
}
int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}
}  // namespace

// Launch choices found by the autotuner, per tree shape (process-wide): a context that
// builds a tree of a shape already tuned starts from that choice without timing.
using ShapeKey = std::tuple<int64_t, int, int, int, bool, bool, bool, int>;
struct LaunchChoice {
    int wpt, occ_pct;
};
std::mutex g_choice_mutex;
std::map<ShapeKey, LaunchChoice> g_choice;

ShapeKey shape_key(const treeray_ctx* c) {
    return ShapeKey(c->nleaves, c->lmax, c->p.npix, c->p.nbins, c->has_thick || c->force_thick, needs_general(c),
                    c->amr, c->device);
}

void apply_cached_launch_choice(treeray_ctx* c) {
    std::lock_guard<std::mutex> lock(g_choice_mutex);
    const auto it = g_choice.find(shape_key(c));
    if (it == g_choice.end()) return;
    c->wpt = it->second.wpt;
    c->occ_pct = it->second.occ_pct;
}

// Times the result-neutral launch choices of the evaluate kernel on a sample of targets:
// warps per target (2, 3, 4, 8; 3 only for thin tiles) at full occupancy, then for the
// fastest team size the resident teams per SM (100, 75, 50 % of those that fit).
treeray_status autotune(treeray_ctx* c, int64_t n_sample, int* best, float* ms, int* best_occ, float* ms_occ,
                        cudaStream_t s) {
    const int64_t N = c->nleaves;
    const int64_t n = std::max<int64_t>(1, std::min(n_sample, N));
    int64_t step = 1000003;
    while (gcd64(step, N) != 1) step += 2;
    int32_t* t = nullptr;
    float* J = nullptr;
    double* F = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    struct Free {
        int32_t*& t;
        float*& J;
        double*& F;
        cudaEvent_t& e0;
        cudaEvent_t& e1;
        ~Free() {
            if (t) cudaFree(t);
            if (J) cudaFree(J);
            if (F) cudaFree(F);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } guard{t, J, F, e0, e1};
    treeray_status rc;
    if ((rc = dev_alloc(c, (void**)&t, sizeof(int32_t) * n)) != TREERAY_OK) return rc;
    if ((rc = dev_alloc(c, (void**)&J, sizeof(float) * n)) != TREERAY_OK) return rc;
    if ((rc = dev_alloc(c, (void**)&F, sizeof(double) * 3 * n)) != TREERAY_OK) return rc;
    TR_CUDA(cudaEventCreate(&e0));
    TR_CUDA(cudaEventCreate(&e1));
    k_sample_targets<<<(int)((n + 255) / 256), 256, 0, s>>>(t, n, N, step);
    ++c->launches;
    const bool thick = c->has_thick || c->force_thick;
    auto time_once = [&](int wpt, float* out) -> treeray_status {
        EvalArgs a = make_args(c, t, n);
        a.J = J;
        a.F = F;
        for (int rep = 0; rep < 2; ++rep) {  // the second launch is timed
            if (rep == 1) TR_CUDA(cudaEventRecord(e0, s));
            const treeray_status r = dispatch_team(c, thick, needs_general(c), wpt, a, nullptr, nullptr, 1, c->lmax, s);
            if (r != TREERAY_OK) return r;
        }
        TR_CUDA(cudaEventRecord(e1, s));
        TR_CUDA(cudaEventSynchronize(e1));
        TR_CUDA(cudaEventElapsedTime(out, e0, e1));
        return TREERAY_OK;
    };
    const int cand[4] = {2, 3, 4, 8};
    float bestt = 0.0f;
    int bw = c->wpt;
    bool first = true;
    c->occ_pct = 100;
    for (int k = 0; k < 4; ++k) {
        // teams of three warps exist for thin tiles below 768 rays only
        if (cand[k] == 3 && (thick || c->p.npix > 192)) {
            if (ms) ms[k] = -1.0f;
            continue;
        }
        float t_ms = 0.0f;
        if ((rc = time_once(cand[k], &t_ms)) != TREERAY_OK) return rc;
        if (ms) ms[k] = t_ms;
        if (first || t_ms < bestt) {
            bestt = t_ms;
            bw = cand[k];
            first = false;
        }
    }
    const int occ[3] = {100, 75, 50};
    int bo = 100;
    if (ms_occ) ms_occ[0] = bestt;
    for (int k = 1; k < 3; ++k) {
        c->occ_pct = occ[k];
        float t_ms = 0.0f;
        rc = time_once(bw, &t_ms);
        c->occ_pct = 100;
        if (rc != TREERAY_OK) return rc;
        if (ms_occ) ms_occ[k] = t_ms;
        if (t_ms < bestt) {
            bestt = t_ms;
            bo = occ[k];
        }
    }
    c->wpt = bw;
    c->occ_pct = bo;
    if (best) *best = bw;
    if (best_occ) *best_occ = bo;
    {
        std::lock_guard<std::mutex> lock(g_choice_mutex);
        g_choice[shape_key(c)] = LaunchChoice{bw, bo};
    }
    return TREERAY_OK;
}

}  // namespace tr

// ----------------------------------------------------------------------- batches
struct treeray_batch {
    // boxes split by the kernel they need (thin only, or with thick material); one
    // persistent launch per non-empty group
    struct Group {
        std::vector<int> box;  // indices into ctx
        std::vector<tr::EvalArgs> desc;
        std::vector<int64_t> start;
        unsigned long long* d_queue = nullptr;
        int max_lmax = 0;
        bool periodic = false;  // some box needs the general kernel (periodic, COL, float thin tiles)
    };
    std::vector<treeray_t> ctx;
    Group g[2];
    std::vector<void*> lastJ, lastF;
    int wpt_thin = 3;  // team size of the thin-tile launch (2, 3 or 4 warps)
    cudaGraphExec_t graph = nullptr;
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

using namespace tr;

extern "C" {

treeray_status treeray_batch_create(const treeray_t* ctxs, int n_boxes, treeray_batch_t* out) {
    if (!ctxs || !out || n_boxes < 1) {
        set_error("batch_create: contexts and n_boxes >= 1 required");
        return TREERAY_EINVAL;
    }
    *out = nullptr;
    const treeray_t c0 = ctxs[0];
    for (int k = 0; k < n_boxes; ++k) {
        const treeray_t c = ctxs[k];
        if (!c || !c->built) {
            set_error("batch_create: every context must hold a built tree");
            return TREERAY_ENOTBUILT;
        }
        if (c->p.npix != c0->p.npix || c->p.nbins != c0->p.nbins || c->device != c0->device) {
            set_error("batch_create: all boxes need the same npix, nbins and device");
            return TREERAY_EINVAL;
        }
    }
    treeray_batch* b = new (std::nothrow) treeray_batch();
    if (!b) {
        set_error("out of host memory");
        return TREERAY_ENOMEM;
    }
    b->ctx.assign(ctxs, ctxs + n_boxes);
    for (int k = 0; k < n_boxes; ++k)  // thin boxes run the team size of the first one's choice
        if (!(ctxs[k]->has_thick || ctxs[k]->force_thick)) {
            b->wpt_thin = (ctxs[k]->wpt == 2 || ctxs[k]->wpt == 3) ? ctxs[k]->wpt : 4;
            break;
        }
    for (int k = 0; k < n_boxes; ++k) {
        treeray_t c = ctxs[k];
        treeray_batch::Group& g = b->g[(c->has_thick || c->force_thick) ? 1 : 0];
        EvalArgs a = make_args(c, nullptr, c->nleaves);
        if (g.start.empty()) g.start.push_back(0);
        g.box.push_back(k);
        g.desc.push_back(a);
        g.start.push_back(g.start.back() + c->nleaves);
        g.max_lmax = std::max(g.max_lmax, c->lmax);
        g.periodic = g.periodic || needs_general(c);
    }
    auto fail = [&](treeray_status rc) {
        treeray_batch_destroy(b);
        return rc;
    };
    for (auto& g : b->g) {
        if (g.box.empty()) continue;
        // the group's launches use its first context's team-stack scratch, for the
        // deepest tree of the group
        const treeray_status rs = reserve_eval_stacks(b->ctx[g.box[0]], g.max_lmax, nullptr);
        if (rs != TREERAY_OK) return fail(rs);
        const treeray_status rt =
            reserve_team_tiles_kind(b->ctx[g.box[0]], g.start.back(), &g == &b->g[1], nullptr);
        if (rt != TREERAY_OK) return fail(rt);
        if (cudaMalloc(&g.d_queue, sizeof(unsigned long long)) != cudaSuccess) {
            set_error("batch_create: device allocation failed");
            return fail(TREERAY_ENOMEM);
        }
    }
    *out = b;
    return TREERAY_OK;
}

treeray_status treeray_batch_destroy(treeray_batch_t b) {
    if (!b) return TREERAY_OK;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    for (auto& g : b->g) {
        if (g.d_queue) cudaFree(g.d_queue);
    }
    delete b;
    return TREERAY_OK;
}

namespace {
treeray_status batch_launch(treeray_batch_t b, cudaStream_t s) {
    for (int t = 0; t < 2; ++t) {
        treeray_batch::Group& g = b->g[t];
        if (g.box.empty()) continue;
        treeray_t c0 = b->ctx[g.box[0]];
        EvalArgs a = g.desc[0];
        a.n = g.start.back();
        a.queue = g.d_queue;
        a.targets = nullptr;
        a.skip = nullptr;
        const treeray_status rc =
            dispatch_team(c0, t == 1, g.periodic, t == 0 ? b->wpt_thin : 4, a, g.desc.data(), g.start.data(),
                          (int)g.box.size(), g.max_lmax, s);
        if (rc != TREERAY_OK) return rc;
    }
    return TREERAY_OK;
}
}  // namespace

treeray_status treeray_batch_evaluate(treeray_batch_t b, float* const* J, double* const* F, int use_graph,
                                      treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_batch_evaluate");
    if (!b || !J || !F) {
        set_error("batch_evaluate: batch, J and F required");
        return TREERAY_EINVAL;
    }
    bool changed = !b->graph;
    for (auto& g : b->g)
        for (size_t q = 0; q < g.box.size(); ++q) {
            const int k = g.box[q];
            if (!J[k] || !F[k]) {
                set_error("batch_evaluate: every box needs J and F");
                return TREERAY_EINVAL;
            }
            changed = changed || g.desc[q].J != J[k] || g.desc[q].F != F[k];
            g.desc[q].J = J[k];
            g.desc[q].F = F[k];
        }
    cudaStream_t us = (cudaStream_t)stream;
    // the descriptors travel as kernel parameters: a captured graph holds the output
    // pointers of its capture and is captured again when they change
    if (changed && b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (!use_graph) return batch_launch(b, us);
    if (!b->gstream) TR_CUDA(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : b->ev)
        if (!e) TR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (!b->graph) {
        cudaGraph_t gr = nullptr;
        TR_CUDA(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
        treeray_status rc = batch_launch(b, b->gstream);
        cudaError_t ce = cudaStreamEndCapture(b->gstream, &gr);
        if (rc != TREERAY_OK) {
            if (gr) cudaGraphDestroy(gr);
            return rc;
        }
        TR_CUDA(ce);
        ce = cudaGraphInstantiate(&b->graph, gr, 0);
        cudaGraphDestroy(gr);
        TR_CUDA(ce);
    }
    TR_CUDA(cudaEventRecord(b->ev[0], us));
    TR_CUDA(cudaStreamWaitEvent(b->gstream, b->ev[0], 0));
    TR_CUDA(cudaGraphLaunch(b->graph, b->gstream));
    b->ctx[0]->launches += 1;
    TR_CUDA(cudaEventRecord(b->ev[1], b->gstream));
    TR_CUDA(cudaStreamWaitEvent(us, b->ev[1], 0));
    return TREERAY_OK;
}

treeray_status treeray_set_warps_per_target(treeray_t c, int wpt) {
    if (!c || (wpt != 2 && wpt != 3 && wpt != 4 && wpt != 8)) {
        set_error("set_warps_per_target: wpt must be 2, 3, 4 or 8");
        return TREERAY_EINVAL;
    }
    c->wpt = wpt;
    return TREERAY_OK;
}

treeray_status treeray_autotune(treeray_t c, int64_t n_sample, int* best_wpt, float* ms,
                                treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_autotune");
    if (!c || !c->built) {
        set_error("autotune: no tree");
        return c ? TREERAY_ENOTBUILT : TREERAY_EINVAL;
    }
    if (n_sample < 1) {
        set_error("autotune: n_sample >= 1");
        return TREERAY_EINVAL;
    }
    return autotune(c, n_sample, best_wpt, ms, nullptr, nullptr, (cudaStream_t)stream);
}

treeray_status treeray_autotune_launch(treeray_t c, int64_t n_sample, int* best_wpt, int* best_occupancy_pct,
                                       float* ms_wpt, float* ms_occupancy, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_autotune_launch");
    if (!c || !c->built) {
        set_error("autotune_launch: no tree");
        return c ? TREERAY_ENOTBUILT : TREERAY_EINVAL;
    }
    if (n_sample < 1) {
        set_error("autotune_launch: n_sample >= 1");
        return TREERAY_EINVAL;
    }
    return autotune(c, n_sample, best_wpt, ms_wpt, best_occupancy_pct, ms_occupancy, (cudaStream_t)stream);
}

treeray_status treeray_get_launch_config(treeray_t c, int* wpt, int* occupancy_pct) {
    if (!c) {
        set_error("get_launch_config: null context");
        return TREERAY_EINVAL;
    }
    if (wpt) *wpt = c->wpt;
    if (occupancy_pct) *occupancy_pct = c->occ_pct;
    return TREERAY_OK;
}

treeray_status treeray_set_occupancy(treeray_t c, int occupancy_pct) {
    if (!c || occupancy_pct < 1 || occupancy_pct > 100) {
        set_error("set_occupancy: occupancy_pct in 1..100");
        return TREERAY_EINVAL;
    }
    c->occ_pct = occupancy_pct;
    return TREERAY_OK;
}

}  // extern "C"
