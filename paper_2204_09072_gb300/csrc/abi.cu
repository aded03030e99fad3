// C ABI of the treeray library: argument checking, context and table management.
// The compute steps live in build.cu, evaluate.cu and post.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <limits>
#include <string>
#include <vector>

#include "internal.h"

namespace tr {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

void free_tables(DeviceTables& t) {
    void* ptrs[] = {t.nhat, t.alpha_off, t.alpha_pair, t.alpha_ent, t.bin_thr, t.bin_thr2, t.R2, t.Rh,
                    t.Rd, t.lvlp, t.open_max, t.str_lo, t.str_hi, t.scal, t.err, t.queue};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    t = DeviceTables{};
}

treeray_status dev_alloc(treeray_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (c && c->alloc_fail_at > 0 && ++c->alloc_count >= c->alloc_fail_at) {
        c->alloc_fail_at = 0;  // one failure per arrangement
        set_error("device allocation failed (injected)");
        return TREERAY_ENOMEM;
    }
    TR_CUDA(cudaMalloc(p, bytes));
    return TREERAY_OK;
}

namespace {
template <typename T>
treeray_status upload(treeray_ctx* c, T** dst, const std::vector<T>& src, cudaStream_t s) {
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    const treeray_status rc = dev_alloc(c, (void**)dst, sizeof(T) * std::max<size_t>(src.size(), 1));
    if (rc != TREERAY_OK) return rc;
    if (!src.empty())
        TR_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s));
    return TREERAY_OK;
}
}  // namespace

// Ray directions n_h (pixel centres), per orientation R_o n_h, rounded to FP32 from FP64.
treeray_status upload_directions(treeray_ctx* c, cudaStream_t s) {
    const int np = c->p.npix;
    const size_t k = std::max<size_t>(1, c->rot.size() / 9);
    std::vector<float> nh(3 * (size_t)np * k);
    for (int h = 0; h < np; ++h) {
        double v[3];
        healpix_pix2vec(c->ht.nside, h, v);
        for (size_t o = 0; o < k; ++o)
            for (int a = 0; a < 3; ++a) {
                double w = v[a];
                if (!c->rot.empty()) {
                    const double* R = c->rot.data() + 9 * o + 3 * a;
                    w = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
                }
                nh[3 * (o * np + h) + a] = (float)w;
            }
    }
    c->ht.nhat = nh;
    treeray_status rc = upload(c, &c->dt.nhat, nh, s);
    if (rc != TREERAY_OK) return rc;
    TR_CUDA(cudaStreamSynchronize(s));  // the host vector is replaced on the next call
    return TREERAY_OK;
}

// The default orientation map of a grid, leaf l -> l mod k, unless the caller's map fits it.
treeray_status ensure_orient_map(treeray_ctx* c, cudaStream_t s) {
    if (c->rot.empty()) return TREERAY_OK;
    if (c->orient && c->orient_n == c->nleaves) return TREERAY_OK;
    const int k = (int)(c->rot.size() / 9);
    std::vector<uint8_t> m((size_t)c->nleaves);
    for (int64_t l = 0; l < c->nleaves; ++l) m[l] = (uint8_t)(l % k);
    c->orient_user = false;
    c->orient_n = 0;
    treeray_status rc = upload(c, &c->orient, m, s);
    if (rc != TREERAY_OK) return rc;
    TR_CUDA(cudaStreamSynchronize(s));
    c->orient_n = c->nleaves;
    return TREERAY_OK;
}

// Per-grid tables: the alpha table (cached by grid shape) and, for every target level,
// the integer thresholds of the walk's decisions:
//   bin i      : d^2 >= ceil(R_i^2)                      (segment index, i >= 1)
//   open       : d^2 <= open_max[level]  <=>  theta^2 d^2 <= E^2 in FP64
//   straddle   : d^2 >= ceil((R_j + s)^2) -> the node's near edge lies beyond R_j;
//                d^2 >= ceil((R_j - s)^2) (0 when R_j <= s) -> its far edge does,
//                s = sqrt(3)/2 E (half the node's diagonal)
namespace {
// (first entry, end) of every key of every orientation: one 8-byte load per accepted node in
// the evaluation instead of two 4-byte ones
__global__ void k_alpha_pairs(const int32_t* off, int2* pair, int64_t keys, int64_t stride, int64_t k) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= keys * k) return;
    const int64_t o = i / keys, key = i - o * keys;
    pair[i] = make_int2(off[o * stride + key], off[o * stride + key + 1]);
}
}  // namespace

treeray_status upload_tables(treeray_ctx* c, cudaStream_t s) {
    const int L = c->lmax, nb = c->p.nbins;
    if (c->tab_lmax == L && c->tab_amr == c->amr) {
        c->built = true;  // tables depend only on the grid shape: reuse
        return ensure_orient_map(c, s);
    }
    {
        c->ht.npix = c->p.npix;
        c->ht.nside = healpix_nside(c->p.npix);
        c->ht.s = c->p.alpha_s;
        if (!build_alpha_table(c->ht, c->p.theta, L, c->amr, c->p.col_mapping != 0, c->rot)) {
            set_error("angular-kernel tables of all orientations exceed 2^31 entries");
            return TREERAY_ENOMEM;
        }
        treeray_status rc;
        if ((rc = upload(c, &c->dt.alpha_off, c->ht.alpha_off, s)) != TREERAY_OK) return rc;
        if ((rc = upload(c, &c->dt.alpha_ent, c->ht.alpha_ent, s)) != TREERAY_OK) return rc;
        const int64_t W = 2 * c->ht.D + 1, keys = W * W * W, stride = keys + 1;
        const int64_t k = (int64_t)c->ht.alpha_off.size() / stride;
        if (c->dt.alpha_pair) cudaFree(c->dt.alpha_pair);
        c->dt.alpha_pair = nullptr;
        if ((rc = dev_alloc(c, (void**)&c->dt.alpha_pair, sizeof(int2) * (size_t)std::max<int64_t>(1, keys * k))) !=
            TREERAY_OK)
            return rc;
        if (keys * k > 0) {
            k_alpha_pairs<<<(unsigned)((keys * k + 255) / 256), 256, 0, s>>>(c->dt.alpha_off, c->dt.alpha_pair, keys,
                                                                             stride, k);
            c->launches += 1;
            TR_CUDA(cudaGetLastError());
        }
    }
    std::vector<int64_t> thr((size_t)(L + 1) * nb), omax(L + 1);
    std::vector<float> R2((size_t)(L + 1) * nb), Rh((size_t)(L + 1) * nb);
    std::vector<double> Rd((size_t)(L + 1) * nb);
    std::vector<float2> lvlp(L + 1);
    std::vector<int64_t> slo((size_t)(L + 1) * (L + 1) * nb), shi(slo.size());
    std::vector<double> R(nb + 1);
    const double th2 = c->p.theta * c->p.theta;
    const int64_t dmax = (int64_t)1 << 62;
    for (int lv = 0; lv <= L; ++lv) {
        const int64_t E = (int64_t)2 << (L - lv);
        const double E2 = (double)(E * E);
        // largest integer d2 with th2 * d2 <= E^2
        int64_t x;
        const double guess = E2 / th2;
        if (!(guess < 4.0e18)) x = dmax;
        else {
            x = (int64_t)std::floor(guess);
            while (x > 0 && th2 * (double)x > E2) --x;
            while (x < dmax && th2 * (double)(x + 1) <= E2) ++x;
        }
        omax[lv] = x;
    }
    for (int lt = 0; lt <= L; ++lt) {
        radii(nb, L, c->p.periodic, c->p.bin_spacing, (int64_t)2 << (L - lt), R.data());
        // segment guess parameters (the integer thresholds decide): geometric radii
        // i ~ log2(d^2 / R_0^2) nb / (2 log2(R_max / R_0)); quadratic radii
        // i ~ sqrt((d - R_0) nb^2 / (R_max - R_0))
        // (the quadratic pair carries -R_0, so the kernel tells the two apart by its sign)
        lvlp[lt] = c->p.bin_spacing == 1
                       ? make_float2((float)-R[0], (float)((double)nb * nb / (R[nb] - R[0])))
                       : make_float2((float)(1.0 / (R[0] * R[0])), (float)(0.5 * nb / std::log2(R[nb] / R[0])));
        for (int i = 0; i < nb; ++i) {
            thr[(size_t)lt * nb + i] = (int64_t)std::ceil(R[i] * R[i]);
            R2[(size_t)lt * nb + i] = (float)(R[i] * R[i]);
            Rh[(size_t)lt * nb + i] = (float)R[i];
            Rd[(size_t)lt * nb + i] = R[i];
        }
        for (int ln = 0; ln <= L; ++ln) {
            const int64_t E = (int64_t)2 << (L - ln);
            const double sd = (std::sqrt(3.0) * 0.5) * (double)E;
            for (int j = 0; j < nb; ++j) {
                const double up = R[j] + sd;
                const double dn = R[j] - sd;
                const size_t q = ((size_t)lt * (L + 1) + ln) * nb + j;
                slo[q] = (int64_t)std::ceil(up * up);
                shi[q] = dn <= 0.0 ? 0 : (int64_t)std::ceil(dn * dn);
            }
        }
    }
    treeray_status rc;
    if ((rc = upload(c, &c->dt.bin_thr, thr, s)) != TREERAY_OK) return rc;
    {  // neighbouring thresholds side by side: one 16-byte load per segment decision
        std::vector<longlong2> thr2(thr.size());
        for (int lt = 0; lt <= L; ++lt)
            for (int i = 0; i < nb; ++i) {
                const size_t k = (size_t)lt * nb + i;
                thr2[k].x = thr[k];
                thr2[k].y = i + 1 < nb ? thr[k + 1] : std::numeric_limits<long long>::max();
            }
        if ((rc = upload(c, &c->dt.bin_thr2, thr2, s)) != TREERAY_OK) return rc;
    }
    if ((rc = upload(c, &c->dt.R2, R2, s)) != TREERAY_OK) return rc;
    if ((rc = upload(c, &c->dt.Rh, Rh, s)) != TREERAY_OK) return rc;
    if ((rc = upload(c, &c->dt.Rd, Rd, s)) != TREERAY_OK) return rc;
    if ((rc = upload(c, &c->dt.open_max, omax, s)) != TREERAY_OK) return rc;
    if ((rc = upload(c, &c->dt.lvlp, lvlp, s)) != TREERAY_OK) return rc;
    if ((rc = upload(c, &c->dt.str_lo, slo, s)) != TREERAY_OK) return rc;
    if ((rc = upload(c, &c->dt.str_hi, shi, s)) != TREERAY_OK) return rc;
    TR_CUDA(cudaStreamSynchronize(s));  // host vectors die on return
    c->tab_lmax = L;
    c->tab_amr = c->amr;
    c->built = true;
    return ensure_orient_map(c, s);
}

}  // namespace tr

using namespace tr;

namespace {
treeray_status check_ctx(treeray_t c, bool need_tree) {
    if (!c) {
        set_error("null context");
        return TREERAY_EINVAL;
    }
    if (need_tree && !c->built) {
        set_error("no tree: call treeray_build first");
        return TREERAY_ENOTBUILT;
    }
    return TREERAY_OK;
}
}  // namespace

extern "C" {

treeray_status treeray_create(const treeray_params* p, treeray_t* out) {
    set_error("");
    if (!p || !out) {
        set_error("null argument");
        return TREERAY_EINVAL;
    }
    *out = nullptr;
    if (p->npix != 12 && p->npix != 48 && p->npix != 192 && p->npix != 768) {
        set_error("npix must be 12, 48, 192 or 768");
        return TREERAY_EINVAL;
    }
    if (p->nbins < 1 || p->nbins > kMaxBins) {
        set_error("nbins must lie in 1..64");
        return TREERAY_EINVAL;
    }
    if (!(p->theta > 0.0 || p->theta < 0.0) || p->theta > 2.0) {
        set_error("theta must lie in (0, 2], or be negative for the ray-matched angle");
        return TREERAY_EINVAL;
    }
    if (p->col_mapping != 0 && p->col_mapping != 1) {
        set_error("col_mapping must be 0 or 1");
        return TREERAY_EINVAL;
    }
    if (p->bin_spacing != 0 && p->bin_spacing != 1) {
        set_error("bin_spacing must be 0 (geometric) or 1 (quadratic)");
        return TREERAY_EINVAL;
    }
    if (p->kappa_model != 0 && p->kappa_model != 1) {
        set_error("kappa_model must be 0 or 1");
        return TREERAY_EINVAL;
    }
    if (p->alpha_s < 4 || p->alpha_s > 16 || p->alpha_s % 4 != 0) {
        set_error("alpha_s must be 4, 8, 12 or 16");
        return TREERAY_EINVAL;
    }
    if (p->periodic < 0 || p->periodic > 7) {
        set_error("periodic must be a mask of axes in 0..7");
        return TREERAY_EINVAL;
    }
    treeray_ctx* c = new (std::nothrow) treeray_ctx();
    if (!c) {
        set_error("out of host memory");
        return TREERAY_ENOMEM;
    }
    c->p = *p;
    // negative theta: the opening angle matched to the ray size (Sec. 7.6)
    if (c->p.theta < 0.0) c->p.theta = std::sqrt(4.0 * kPi / (double)p->npix);
    cudaGetDevice(&c->device);
    c->ht.npix = p->npix;
    c->ht.nside = healpix_nside(p->npix);
    c->ht.s = p->alpha_s;
    auto fail = [&](treeray_status rc) {
        free_tables(c->dt);
        delete c;
        return rc;
    };
    treeray_status rc = upload_directions(c, nullptr);
    if (rc != TREERAY_OK) return fail(rc);
    if (cudaMalloc(&c->dt.scal, sizeof(double) * 4) != cudaSuccess ||
        cudaMalloc(&c->dt.err, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&c->dt.queue, sizeof(unsigned long long)) != cudaSuccess) {
        set_error("device allocation failed");
        return fail(TREERAY_ENOMEM);
    }
    if (cudaMemset(c->dt.err, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        set_error("device initialisation failed");
        return fail(TREERAY_ECUDA);
    }
    *out = c;
    return TREERAY_OK;
}

treeray_status treeray_destroy(treeray_t c) {
    if (!c) return TREERAY_OK;
    if (c->fp_Tnew) cudaFree(c->fp_Tnew);
    if (c->fp_J) cudaFree(c->fp_J);
    if (c->fp_F) cudaFree(c->fp_F);
    if (c->fp_flags) cudaFree(c->fp_flags);
    if (c->stack_scr) cudaFree(c->stack_scr);
    if (c->gtile) cudaFree(c->gtile);
    if (c->orient) cudaFree(c->orient);
    if (c->fp_stream) cudaStreamDestroy(c->fp_stream);
    for (cudaEvent_t e : c->fp_ev)
        if (e) cudaEventDestroy(e);
    free_tree(c->tree);
    free_tables(c->dt);
    delete c;
    return TREERAY_OK;
}

treeray_status treeray_build(treeray_t c, const treeray_grid* g, const float* rho, const float* Td,
                             const float* kappa, int n_stars, const double* star_pos,
                             const double* star_lum, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_build");
    treeray_status rc = check_ctx(c, false);
    if (rc != TREERAY_OK) return rc;
    if (!g) {
        set_error("null grid");
        return TREERAY_EINVAL;
    }
    rc = build_tree(c, g, rho, Td, kappa, n_stars, star_pos, star_lum, (cudaStream_t)stream);
    if (rc != TREERAY_OK) return rc;
    rc = reserve_eval_stacks(c, c->lmax, (cudaStream_t)stream);
    if (rc == TREERAY_OK) rc = reserve_team_tiles(c, c->nleaves, (cudaStream_t)stream);
    if (rc != TREERAY_OK) c->built = false;  // a failed build leaves no usable tree
    return rc;
}

treeray_status treeray_set_orientations(treeray_t c, int k, const double* rot, const uint8_t* orient) {
    NvtxRange nvtx_("treeray_set_orientations");
    treeray_status rc = check_ctx(c, orient != nullptr);
    if (rc != TREERAY_OK) return rc;
    if (k < 0 || k > kMaxOrientations || (k > 0 && !rot) || (k == 0 && orient)) {
        set_error("set_orientations: k in 0..64, rot required for k > 0, no map for k = 0");
        return TREERAY_EINVAL;
    }
    for (int o = 0; o < k; ++o) {
        const double* R = rot + 9 * o;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const double d = R[3 * a] * R[3 * b] + R[3 * a + 1] * R[3 * b + 1] + R[3 * a + 2] * R[3 * b + 2];
                if (!(std::fabs(d - (a == b ? 1.0 : 0.0)) <= 1e-9)) {
                    set_error("set_orientations: rotation " + std::to_string(o) + " is not orthonormal");
                    return TREERAY_EINVAL;
                }
            }
        const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                           R[2] * (R[3] * R[7] - R[4] * R[6]);
        if (!(det > 0.0)) {
            set_error("set_orientations: rotation " + std::to_string(o) + " is a reflection");
            return TREERAY_EINVAL;
        }
    }
    std::vector<uint8_t> m;
    if (orient) {  // checked on the host: every value < k
        m.resize((size_t)c->nleaves);
        TR_CUDA(cudaMemcpy(m.data(), orient, m.size(), cudaMemcpyDeviceToHost));
        for (uint8_t v : m)
            if ((int)v >= k) {
                set_error("set_orientations: map value " + std::to_string((int)v) + " >= k");
                return TREERAY_EINVAL;
            }
    }
    TR_CUDA(cudaDeviceSynchronize());  // no launch may still read the old tables
    c->rot.assign(rot ? rot : nullptr, rot ? rot + 9 * (size_t)k : nullptr);
    if (c->orient) cudaFree(c->orient);
    c->orient = nullptr;
    c->orient_n = 0;
    c->orient_user = false;
    if ((rc = upload_directions(c, nullptr)) != TREERAY_OK) return rc;
    if (orient) {
        if ((rc = upload(c, &c->orient, m, nullptr)) != TREERAY_OK) return rc;
        TR_CUDA(cudaDeviceSynchronize());
        c->orient_n = c->nleaves;
        c->orient_user = true;
    }
    c->tab_lmax = -1;  // the angular-kernel tables follow the orientations
    if (!c->built) return TREERAY_OK;
    return upload_tables(c, nullptr);
}

treeray_status treeray_evaluate(treeray_t c, const int32_t* targets, int64_t n, float* J, double* F,
                                treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_evaluate");
    treeray_status rc = check_ctx(c, true);
    if (rc != TREERAY_OK) return rc;
    if (n == 0 && targets == nullptr && c->nleaves != 0) return TREERAY_OK;  // an empty target list
    if (!J || !F || n < 0 || (!targets && n != c->nleaves)) {
        set_error("evaluate: J and F required; n must equal the leaf count when targets is NULL");
        return TREERAY_EINVAL;
    }
    if (n == 0) return TREERAY_OK;
    return launch_evaluate(c, targets, n, J, F, (cudaStream_t)stream);
}

treeray_status treeray_radpressure(treeray_t c, const float* J, const double* F, float* u, float* a_rp,
                                   float* force, float* p_src, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_radpressure");
    treeray_status rc = check_ctx(c, true);
    if (rc != TREERAY_OK) return rc;
    if (!J || !F) {
        set_error("radpressure: J and F required");
        return TREERAY_EINVAL;
    }
    return launch_radpressure(c, J, F, u, a_rp, force, p_src, (cudaStream_t)stream);
}

treeray_status treeray_uv_radpressure(treeray_t c, const float* nph, const float* uph, const float* x_ion,
                                      float* a_uv, float* force_uv, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_uv_radpressure");
    treeray_status rc = check_ctx(c, true);
    if (rc != TREERAY_OK) return rc;
    if (!nph || !uph) {
        set_error("uv_radpressure: nph and uph required");
        return TREERAY_EINVAL;
    }
    return launch_uv_radpressure(c, nph, uph, x_ion, a_uv, force_uv, (cudaStream_t)stream);
}

treeray_status treeray_dust_temperature(treeray_t c, const float* Tgas, const float* heat_extra,
                                        const float* J, float* Td, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_dust_temperature");
    treeray_status rc = check_ctx(c, true);
    if (rc != TREERAY_OK) return rc;
    if (!Tgas || !J || !Td) {
        set_error("dust_temperature: Tgas, J and Td required");
        return TREERAY_EINVAL;
    }
    return launch_dust(c, Tgas, heat_extra, J, Td, (cudaStream_t)stream);
}

treeray_status treeray_refresh(treeray_t c, const float* Td, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_refresh");
    treeray_status rc = check_ctx(c, true);
    if (rc != TREERAY_OK) return rc;
    if (!Td) {
        set_error("refresh: Td required");
        return TREERAY_EINVAL;
    }
    if (c->p.kappa_model == 1) c->force_thick = true;
    return refresh_tree(c, Td, nullptr, (cudaStream_t)stream);
}

namespace {
// one fixed-point iteration: T_d -> tree moments -> J -> T_new -> largest change, T_d <- T_new
treeray_status fp_iteration(treeray_t c, const float* Tgas, const float* heat, float* Td, double tol,
                            int max_iter, cudaStream_t s) {
    const int* skip = c->fp_flags;
    treeray_status rc;
    if ((rc = refresh_tree(c, Td, skip, s)) != TREERAY_OK) return rc;
    if ((rc = launch_evaluate_skip(c, c->fp_J, c->fp_F, skip, s)) != TREERAY_OK) return rc;
    if ((rc = launch_dust_skip(c, Tgas, heat, c->fp_J, c->fp_Tnew, skip, s)) != TREERAY_OK) return rc;
    return launch_fp_update(c, c->fp_Tnew, Td, tol, max_iter, s);
}
}  // namespace

treeray_status treeray_fixed_point(treeray_t c, const float* Tgas, const float* heat_extra, float* Td,
                                   int max_iter, double tol, int unroll, int* iters,
                                   treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_fixed_point");
    treeray_status rc = check_ctx(c, true);
    if (rc != TREERAY_OK) return rc;
    if (!Tgas || !Td || max_iter < 1 || !(tol > 0.0) || unroll < 0 || unroll > 64) {
        set_error("fixed_point: Tgas and Td required, max_iter >= 1, tol > 0, unroll in 0..64");
        return TREERAY_EINVAL;
    }
    const int64_t N = c->nleaves;
    if (c->fp_cap < N) {
        if (c->fp_Tnew) cudaFree(c->fp_Tnew);
        if (c->fp_J) cudaFree(c->fp_J);
        if (c->fp_F) cudaFree(c->fp_F);
        c->fp_Tnew = nullptr;
        c->fp_J = nullptr;
        c->fp_F = nullptr;
        c->fp_cap = 0;
        if ((rc = dev_alloc(c, (void**)&c->fp_Tnew, sizeof(float) * N)) != TREERAY_OK ||
            (rc = dev_alloc(c, (void**)&c->fp_J, sizeof(float) * N)) != TREERAY_OK ||
            (rc = dev_alloc(c, (void**)&c->fp_F, sizeof(double) * 3 * N)) != TREERAY_OK)
            return rc;
        c->fp_cap = N;
    }
    if (!c->fp_flags && (rc = dev_alloc(c, (void**)&c->fp_flags, sizeof(int) * 4)) != TREERAY_OK) return rc;
    if (!c->fp_stream) TR_CUDA(cudaStreamCreateWithFlags(&c->fp_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : c->fp_ev)
        if (!e) TR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (c->p.kappa_model == 1) c->force_thick = true;
    cudaStream_t us = (cudaStream_t)stream, fs = c->fp_stream;
    TR_CUDA(cudaMemsetAsync(c->fp_flags, 0, sizeof(int) * 4, us));
    TR_CUDA(cudaEventRecord(c->fp_ev[0], us));
    TR_CUDA(cudaStreamWaitEvent(fs, c->fp_ev[0], 0));
    int host_flags[2] = {0, 0};
    if (unroll > 0) {
        // a CUDA graph of `unroll` iterations, replayed until the device flag stops it;
        // iterations after convergence return at once, so the result equals a plain loop
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        TR_CUDA(cudaStreamBeginCapture(fs, cudaStreamCaptureModeThreadLocal));
        for (int u = 0; u < unroll && rc == TREERAY_OK; ++u) rc = fp_iteration(c, Tgas, heat_extra, Td, tol, max_iter, fs);
        cudaError_t ce = cudaStreamEndCapture(fs, &graph);
        if (rc != TREERAY_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        TR_CUDA(ce);
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        TR_CUDA(ce);
        const int launches = (max_iter + unroll - 1) / unroll;
        for (int k = 0; k < launches; ++k) {
            ce = cudaGraphLaunch(exec, fs);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(host_flags, c->fp_flags, sizeof(int) * 2,
                                                         cudaMemcpyDeviceToHost, fs);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(fs);
            if (ce != cudaSuccess || host_flags[0]) break;
        }
        cudaGraphExecDestroy(exec);
        TR_CUDA(ce);
    } else {
        for (int k = 0; k < max_iter; ++k) {
            if ((rc = fp_iteration(c, Tgas, heat_extra, Td, tol, max_iter, fs)) != TREERAY_OK) return rc;
            TR_CUDA(cudaMemcpyAsync(host_flags, c->fp_flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, fs));
            TR_CUDA(cudaStreamSynchronize(fs));
            if (host_flags[0]) break;
        }
    }
    TR_CUDA(cudaEventRecord(c->fp_ev[1], fs));
    TR_CUDA(cudaStreamWaitEvent(us, c->fp_ev[1], 0));
    if (iters) *iters = host_flags[1];
    if (host_flags[0] != 1) {
        set_error("fixed_point: no convergence within max_iter");
        return TREERAY_ENOCONV;
    }
    return TREERAY_OK;
}

treeray_status treeray_check(treeray_t c, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_check");
    treeray_status rc = check_ctx(c, false);
    if (rc != TREERAY_OK) return rc;
    TR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    TR_CUDA(cudaGetLastError());
    unsigned e = 0;
    TR_CUDA(cudaMemcpy(&e, c->dt.err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (e) {
        TR_CUDA(cudaMemset(c->dt.err, 0, sizeof(unsigned)));
        std::string m = "device error:";
        if (e & kErrStack) m += " walk stack overflow;";
        if (e & kErrAlphaKey) m += " angular-kernel key outside the table;";
        if (e & kErrOctree) m += " leaves do not form a complete octree;";
        if (e & kErrTarget) m += " target index out of range;";
        if (e & kErrInput) m += " an input field holds a negative or non-finite value;";
        set_error(m);
        return (e & (kErrTarget | kErrInput)) ? TREERAY_EINVAL : TREERAY_ETIMEOUT;
    }
    return TREERAY_OK;
}

int64_t treeray_leaf_count(treeray_t c) { return c && c->built ? c->nleaves : 0; }
int64_t treeray_node_count(treeray_t c) { return c && c->built ? c->nnodes : 0; }

treeray_status treeray_tree_export(treeray_t c, int32_t* level, int32_t* leaf, int32_t* child0,
                                   int64_t* centre, double* vals, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_tree_export");
    treeray_status rc = check_ctx(c, true);
    if (rc != TREERAY_OK) return rc;
    const int64_t nn = c->nnodes;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int4> geo(nn);
    std::vector<int32_t> perm(c->nleaves);
    std::vector<double> mom(11 * (size_t)nn);
    TR_CUDA(cudaMemcpyAsync(geo.data(), c->tree.geo, sizeof(int4) * nn, cudaMemcpyDeviceToHost, s));
    TR_CUDA(cudaMemcpyAsync(perm.data(), c->tree.perm, sizeof(int32_t) * c->nleaves, cudaMemcpyDeviceToHost, s));
    TR_CUDA(cudaMemcpyAsync(mom.data(), c->tree.mom, sizeof(double) * 11 * nn, cudaMemcpyDeviceToHost, s));
    TR_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < nn; ++i) {
        const int4 g = geo[i];
        if (level) level[i] = g.z >> 24;
        if (leaf) leaf[i] = g.w < 0 ? perm[-1 - g.w] : -1;
        if (child0) child0[i] = g.w < 0 ? -1 : g.w;
        if (centre) {
            centre[3 * i] = g.x;
            centre[3 * i + 1] = g.y;
            centre[3 * i + 2] = g.z & 0xffffff;
        }
        if (vals)
            for (int q = 0; q < 11; ++q) vals[11 * i + q] = mom[(size_t)q * nn + i];
    }
    return TREERAY_OK;
}

treeray_status treeray_leaf_export(treeray_t c, double* kappa, double* tau, double* jsrc, double* psrc,
                                   int32_t* thick, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_leaf_export");
    treeray_status rc = check_ctx(c, true);
    if (rc != TREERAY_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)c->nleaves;
    if (kappa) TR_CUDA(cudaMemcpyAsync(kappa, c->tree.kap, 8 * n, cudaMemcpyDeviceToHost, s));
    if (tau) TR_CUDA(cudaMemcpyAsync(tau, c->tree.tau, 8 * n, cudaMemcpyDeviceToHost, s));
    if (jsrc) TR_CUDA(cudaMemcpyAsync(jsrc, c->tree.jsrc, 8 * n, cudaMemcpyDeviceToHost, s));
    if (psrc) TR_CUDA(cudaMemcpyAsync(psrc, c->tree.psrc, 8 * n, cudaMemcpyDeviceToHost, s));
    if (thick) TR_CUDA(cudaMemcpyAsync(thick, c->tree.thickflag, 4 * n, cudaMemcpyDeviceToHost, s));
    TR_CUDA(cudaStreamSynchronize(s));
    return TREERAY_OK;
}

treeray_status treeray_accepted(treeray_t c, const int32_t* targets, int64_t n, int32_t cap,
                                int32_t* counts, int32_t* ids, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_accepted");
    treeray_status rc = check_ctx(c, true);
    if (rc != TREERAY_OK) return rc;
    if (n == 0 && cap >= 1) return TREERAY_OK;  // an empty target list
    if (!targets || !counts || !ids || n < 0 || cap < 1) {
        set_error("accepted: targets, counts, ids and cap >= 1 required");
        return TREERAY_EINVAL;
    }
    return launch_accepted(c, targets, n, cap, counts, ids, (cudaStream_t)stream);
}

treeray_status treeray_walk_stats(treeray_t c, const int32_t* targets, int64_t n, int64_t* totals,
                                  treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_walk_stats");
    treeray_status rc = check_ctx(c, true);
    if (rc != TREERAY_OK) return rc;
    if (n == 0 && targets == nullptr && c->nleaves != 0) return TREERAY_OK;  // an empty target list
    if (!totals || n < 0 || (!targets && n != c->nleaves)) {
        set_error("walk_stats: totals required; n must equal the leaf count when targets is NULL");
        return TREERAY_EINVAL;
    }
    if (n == 0) return TREERAY_OK;
    return launch_walk_stats(c, targets, n, totals, (cudaStream_t)stream);
}

treeray_status treeray_alpha_counts_host(int npix, int s, const int64_t* K, int32_t* counts) {
    if (healpix_nside(npix) < 0 || s < 4 || s % 4 != 0 || !K || !counts) {
        set_error("alpha_counts_host: bad arguments");
        return TREERAY_EINVAL;
    }
    alpha_counts(npix, s, K, counts);
    return TREERAY_OK;
}

treeray_status treeray_alpha_counts_rotated_host(int npix, int s, const int64_t* K, const double* rot,
                                                 int32_t* counts) {
    if (healpix_nside(npix) < 0 || s < 4 || s % 4 != 0 || !K || !rot || !counts) {
        set_error("alpha_counts_rotated_host: bad arguments");
        return TREERAY_EINVAL;
    }
    alpha_counts(npix, s, K, counts, rot);
    return TREERAY_OK;
}

int64_t treeray_kernel_launches(treeray_t c) { return c ? c->launches : 0; }

treeray_status treeray_set_walk_stack_limit(treeray_t c, int entries) {
    treeray_status rc = check_ctx(c, false);
    if (rc != TREERAY_OK) return rc;
    if (entries < 0) {
        set_error("set_walk_stack_limit: entries >= 0");
        return TREERAY_EINVAL;
    }
    c->stack_limit = entries;
    return TREERAY_OK;
}

treeray_status treeray_inject_alloc_failure(treeray_t c, int n) {
    treeray_status rc = check_ctx(c, false);
    if (rc != TREERAY_OK) return rc;
    if (n < 0) {
        set_error("inject_alloc_failure: n >= 0");
        return TREERAY_EINVAL;
    }
    c->alloc_fail_at = n;
    c->alloc_count = 0;
    return TREERAY_OK;
}

const char* treeray_last_error(void) { return g_err.c_str(); }

}  // extern "C"
