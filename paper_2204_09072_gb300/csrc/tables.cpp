// Host-side tables of the treeray library, built once per context and grid shape in
// FP64: HEALPix ray directions, the angular kernel alpha (Sec. 4.2, "Ray mapping"),
// evaluation radii, bin/opening/straddle thresholds.
//
// Every discrete decision the GPU walk makes (open or accept a node, segment index,
// angular-kernel key, straddled segment boundaries) is reduced here to an integer
// threshold on the squared centre distance d^2 in half-cells of the finest level,
// so the kernels decide in exact integer arithmetic.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>

#include "internal.h"

namespace tr {

// ---------------------------------------------------------------- HEALPix
// Nested pixelisation of Gorski et al. (2005): 12 base faces of nside^2 pixels whose
// in-face coordinates (ix, iy) are bit-interleaved. The steps (polar caps against the
// equatorial belt, the face from the two edge indices, the ring shift, the base-face row
// and column tables) follow the standard published algorithm, as the HEALPix library's
// nested ang2pix / pix2vec implement it.
namespace {
constexpr int kFaceRing[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
constexpr int kFacePhi[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

inline int64_t spread_bits(int64_t v) {  // bit b of v -> bit 2b
    int64_t out = 0;
    for (int b = 0; v >> b; ++b) out |= ((v >> b) & 1) << (2 * b);
    return out;
}
inline int64_t gather_bits(int64_t v) {  // bit 2b of v -> bit b
    int64_t out = 0;
    for (int b = 0; (v >> (2 * b)) != 0; ++b) out |= ((v >> (2 * b)) & 1) << b;
    return out;
}
}  // namespace

int healpix_nside(int npix) {
    for (int ns = 1; ns <= 64; ns *= 2)
        if (12 * ns * ns == npix) return ns;
    return -1;
}

int healpix_ang2pix(int nside, double x, double y, double z) {
    const int64_t ns = nside;
    const double r = std::sqrt(x * x + y * y + z * z);
    const double cosT = z / r;
    const double absZ = std::fabs(cosT);
    double phi = std::atan2(y, x);
    if (phi < 0.0) phi += 2.0 * kPi;
    double t = phi * (2.0 / kPi);  // longitude in quarter turns, [0, 4)
    if (t >= 4.0) t -= 4.0;
    int64_t face, ix, iy;
    if (absZ <= 2.0 / 3.0) {  // equatorial belt
        const double a = (double)ns * (0.5 + t);
        const double b = (double)ns * (cosT * 0.75);
        const int64_t jp = (int64_t)(a - b);  // ascending edge index
        const int64_t jm = (int64_t)(a + b);  // descending edge index
        const int64_t fp = jp / ns, fm = jm / ns;
        face = (fp == fm) ? (fp | 4) : (fp < fm ? fp : fm + 8);
        ix = jm & (ns - 1);
        iy = ns - (jp & (ns - 1)) - 1;
    } else {  // polar caps
        int64_t q = (int64_t)t;
        if (q > 3) q = 3;
        const double tp = t - (double)q;
        const double s3 = 3.0 * ((x * x + y * y) / (r * (r + std::fabs(z))));  // 3 (1 - |cos|)
        const double w = (double)ns * std::sqrt(s3);
        int64_t jp = (int64_t)(tp * w);
        int64_t jm = (int64_t)((1.0 - tp) * w);
        jp = std::min(jp, ns - 1);
        jm = std::min(jm, ns - 1);
        if (cosT >= 0) {
            face = q;
            ix = ns - jm - 1;
            iy = ns - jp - 1;
        } else {
            face = q + 8;
            ix = jp;
            iy = jm;
        }
    }
    return (int)(face * ns * ns + (spread_bits(ix) | (spread_bits(iy) << 1)));
}

void healpix_pix2vec(int nside, int pix, double* v) {
    const int64_t ns = nside, nf = ns * ns;
    const int64_t face = pix / nf, in = pix % nf;
    const int64_t ix = gather_bits(in), iy = gather_bits(in >> 1);
    const int64_t ring = kFaceRing[face] * ns - (ix + iy) - 1;  // 1 .. 4 nside - 1 from north
    int64_t nr, shift;
    double z;
    if (ring < ns) {
        nr = ring;
        z = 1.0 - (double)(nr * nr) / (3.0 * (double)nf);
        shift = 0;
    } else if (ring > 3 * ns) {
        nr = 4 * ns - ring;
        z = (double)(nr * nr) / (3.0 * (double)nf) - 1.0;
        shift = 0;
    } else {
        nr = ns;
        z = (double)(2 * ns - ring) * 2.0 / (3.0 * (double)ns);
        shift = (ring - ns) & 1;
    }
    int64_t jp = (kFacePhi[face] * nr + ix - iy + 1 + shift) / 2;
    if (jp > 4 * ns) jp -= 4 * ns;
    if (jp < 1) jp += 4 * ns;
    const double phi = ((double)jp - 0.5 * (double)(shift + 1)) * (kPi / 2.0) / (double)nr;
    const double st = std::sqrt((1.0 - z) * (1.0 + z));
    v[0] = st * std::cos(phi);
    v[1] = st * std::sin(phi);
    v[2] = z;
}

// ---------------------------------------------------------- angular kernel
// alpha for a node at quantised offset K (units of 1/8 of its edge) from the target:
// the s^3 sub-cube centres of the node, seen from the target along
// (2 s K / 8 + 2 a + 1 - s) for a = 0..s-1 per axis, counted per pixel.
// rot (row-major R, may be null): a turned ray set (Sec. 7.6), whose ray h points along
// R n_h; a direction v then counts for ray h when R^T v lies in pixel h.
void alpha_counts(int npix, int s, const int64_t* K, int32_t* counts, const double* rot) {
    const int ns = healpix_nside(npix);
    std::fill(counts, counts + npix, 0);
    const int64_t bx = 2 * s * K[0] / 8 + 1 - s;
    const int64_t by = 2 * s * K[1] / 8 + 1 - s;
    const int64_t bz = 2 * s * K[2] / 8 + 1 - s;
    for (int c = 0; c < s; ++c)
        for (int b = 0; b < s; ++b)
            for (int a = 0; a < s; ++a) {
                const double vx = (double)(bx + 2 * a), vy = (double)(by + 2 * b), vz = (double)(bz + 2 * c);
                if (!rot) {
                    counts[healpix_ang2pix(ns, vx, vy, vz)]++;
                    continue;
                }
                // R^T v, each component summed in the order of the vector's axes
                const double wx = rot[0] * vx + rot[3] * vy + rot[6] * vz;
                const double wy = rot[1] * vx + rot[4] * vy + rot[7] * vz;
                const double wz = rot[2] * vx + rot[5] * vy + rot[8] * vz;
                counts[healpix_ang2pix(ns, wx, wy, wz)]++;
            }
}

namespace {
// Parity class of a key component: 0 -> multiple of 8, 3 -> 4 mod 8, 1 -> 2 mod 4, 2 -> odd.
inline int key_class(int64_t k) {
    int64_t m = ((k % 8) + 8) % 8;
    if (m == 0) return 0;
    if (m == 4) return 3;
    if (m == 2 || m == 6) return 1;
    return 2;
}
}  // namespace

// Keys reachable by the walk: same-level leaves (class 0) anywhere in the cube; nodes
// two or more levels coarser than the target (odd keys) and one level coarser (2 mod 4)
// only when accepted by the opening criterion, i.e. at 8 d / E > 8 / theta, unless the
// grid is AMR (coarser and finer leaves next to the target, classes 1-3 anywhere).
namespace {
// tables already built in this process, keyed by (npix, samples, theta, D, amr, col,
// rotations)
std::mutex g_tab_mutex;
std::map<std::tuple<int, int, double, int64_t, bool, bool, std::vector<double>>,
         std::pair<std::vector<int32_t>, std::vector<uint32_t>>>
    g_tab_cache;
}  // namespace

// col: nodes may be mapped at their centre of luminosity, which moves a key by up to 4
// per axis and gives odd keys at any distance.
// rot: k row-major rotations (k = 0: the unturned grid alone). Orientation o's offsets
// are alpha_off[o (W^3 + 1) + key], all pointing into one shared entry array.
bool build_alpha_table(HostTables& t, double theta, int lmax, bool amr, bool col, const std::vector<double>& rot) {
    const double th = theta > 1e-6 ? theta : 1e-6;
    const double reach = std::max(2.0 / th, std::sqrt(3.0)) + 0.5 * std::sqrt(3.0);
    const int64_t extra = col ? 4 : 0;
    int64_t D = (int64_t)std::ceil(8.0 * reach) + 1 + extra;
    const int64_t cap = 8 * ((int64_t)1 << lmax) + 1 + extra;
    D = std::min(D, cap);
    D = std::min<int64_t>(D, 160 + extra);  // covers the ray-matched angle at 768 rays (D = 133)
    t.D = (int)D;
    const auto key = std::make_tuple(t.npix, t.s, theta, D, amr, col, rot);
    {
        std::lock_guard<std::mutex> lock(g_tab_mutex);
        auto it = g_tab_cache.find(key);
        if (it != g_tab_cache.end()) {
            t.alpha_off = it->second.first;
            t.alpha_ent = it->second.second;
            return true;
        }
    }
    const int64_t W = 2 * D + 1, nk = W * W * W;
    const int64_t norient = std::max<int64_t>(1, (int64_t)(rot.size() / 9));
    const double shell = std::max(0.0, 8.0 / th - std::sqrt(3.0));
    const double shell2 = shell * shell;
    // which keys get an entry
    std::vector<int64_t> keys;
    for (int64_t z = -D; z <= D; ++z)
        for (int64_t y = -D; y <= D; ++y)
            for (int64_t x = -D; x <= D; ++x) {
                const int c = key_class(x);
                if (key_class(y) != c || key_class(z) != c) continue;
                if (x == 0 && y == 0 && z == 0) continue;  // own cell, uniform weights
                if (!amr) {
                    if (c == 3) continue;
                    if ((c == 1 || (c == 2 && !col)) && (double)(x * x + y * y + z * z) < shell2) continue;
                }
                keys.push_back(((z + D) * W + (y + D)) * W + (x + D));
            }
    const size_t nkeys = keys.size();
    std::vector<std::vector<uint32_t>> lists(nkeys * norient);
    const int nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int w = 0; w < nth; ++w)
        pool.emplace_back([&, w]() {
            std::vector<int32_t> cnt(t.npix);
            for (size_t j = w; j < nkeys * norient; j += nth) {
                const size_t q = j % nkeys, o = j / nkeys;
                const int64_t idx = keys[q];
                const int64_t K[3] = {idx % W - D, (idx / W) % W - D, idx / (W * W) - D};
                alpha_counts(t.npix, t.s, K, cnt.data(), rot.empty() ? nullptr : rot.data() + 9 * o);
                for (int h = 0; h < t.npix; ++h)
                    if (cnt[h] > 0) lists[j].push_back((uint32_t)h | ((uint32_t)cnt[h] << 16));
            }
        });
    for (auto& th_ : pool) th_.join();
    // offsets per orientation, one running count over all of them (int32: checked)
    std::vector<int32_t> off((size_t)norient * (nk + 1), 0);
    int64_t run = 0;
    std::vector<int32_t> len(nk);
    for (int64_t o = 0; o < norient; ++o) {
        std::fill(len.begin(), len.end(), 0);
        for (size_t q = 0; q < nkeys; ++q) len[keys[q]] = (int32_t)lists[o * nkeys + q].size();
        int32_t* oo = off.data() + o * (nk + 1);
        for (int64_t i = 0; i <= nk; ++i) {
            if (run > INT32_MAX) return false;
            oo[i] = (int32_t)run;
            if (i < nk) run += len[i];
        }
    }
    std::vector<uint32_t> ent((size_t)run, 0);
    for (int64_t o = 0; o < norient; ++o)
        for (size_t q = 0; q < nkeys; ++q)
            std::copy(lists[o * nkeys + q].begin(), lists[o * nkeys + q].end(),
                      ent.begin() + off[o * (nk + 1) + keys[q]]);
    t.alpha_off.swap(off);
    t.alpha_ent.swap(ent);
    std::lock_guard<std::mutex> lock(g_tab_mutex);
    if (g_tab_cache.size() > 16) g_tab_cache.clear();
    g_tab_cache[key] = std::make_pair(t.alpha_off, t.alpha_ent);
    return true;
}

// R_i = R_0 (R_max / R_0)^(i / nbins), R_0 = Et / 2, R_max = sqrt(3) box (half-cells); with
// periodic axes R_max is the largest closest-copy distance (half the box on those axes)
// (spacing 1: R_i = R_0 + (R_max - R_0) (i / nbins)^2, radii growing quadratically)
void radii(int nbins, int lmax, int periodic, int spacing, int64_t Et, double* R) {
    const double R0 = 0.5 * (double)Et;
    const double B = (double)((int64_t)2 << lmax);
    double Rmax = std::sqrt(3.0) * B;
    if (periodic) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double e = ((periodic >> a) & 1) ? 0.5 * B : B;
            s += e * e;
        }
        Rmax = std::sqrt(s);
    }
    if (spacing == 1) {
        for (int i = 0; i <= nbins; ++i) {
            const double q = (double)i / (double)nbins;
            R[i] = R0 + (Rmax - R0) * (q * q);
        }
        return;
    }
    for (int i = 0; i <= nbins; ++i) R[i] = R0 * std::pow(Rmax / R0, (double)i / (double)nbins);
}

}  // namespace tr
