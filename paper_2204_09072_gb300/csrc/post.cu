// Per-leaf epilogues: radiation energy density and pressure (Sec. 4.5) and the
// equilibrium dust temperature (Sec. 4.6, App. D). Elementwise kernels; the dust balance is
// decided in FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace tr {
namespace {

struct RpArgs {
    const float* J;
    const double* F;
    const double* kap;
    const double* tau;
    const double* psrc;
    const float* rho;
    const int4* geo;
    const int32_t* leaf_node;
    const int32_t* inv_perm;
    float *u, *a, *f, *p;
    int64_t n;
    double box;
};

// u = 4 pi J / c; P_dot = (F/c) kappa rho g(tau) dV with g = (1 - e^-tau)/tau (1 for tau < 1e-4);
// a_RP = P_dot / (rho dV) = (F/c) kappa g
__global__ void k_radpressure(RpArgs r) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= r.n) return;
    const int lvl = r.geo[r.leaf_node[r.inv_perm[k]]].z >> 24;
    const double dx = ldexp(r.box, -lvl);
    const double dV = (dx * dx) * dx;
    const double tau = r.tau[k];
    // g in FP32 (the outputs are FP32); 1/c as a constant factor: no FP64 divisions
    const float tf = (float)tau;
    const double g = tau < 1e-4 ? 1.0 : (double)(-expm1f(-tf) / tf);
    const double kap = r.kap[k];
    const double kr = kap * (double)r.rho[k];
    constexpr double inv_c = 1.0 / kLightC;
    if (r.u) r.u[k] = (float)((4.0 * kPi * inv_c) * (double)r.J[k]);
    for (int ax = 0; ax < 3; ++ax) {
        const double Fc = r.F[3 * k + ax] * inv_c;
        if (r.f) r.f[3 * k + ax] = (float)(Fc * kr * g * dV);
        if (r.a) r.a[3 * k + ax] = (float)(Fc * kap * g);
    }
    if (r.p) r.p[k] = (float)r.psrc[k];
}

// Radiation pressure of the ionising (UV) radiation (App. C) on dust, neutral and ionised
// hydrogen, from a given photon flux N (photons/s/cm^2), its unit direction u and the
// ionised fraction x (NULL: 1):
//   P_dot = (E/c) [sigma_d n N + sigma_H (1 - x) n N + alpha_B (x n)^2] u dV, n = X rho / m_H,
// E = 18 eV, sigma_d = 1.5e-21 cm^2 per H, alpha_B = 2.5e-13 cm^3/s, sigma_H = 6.3e-18 cm^2
// (the Lyman-edge cross-section: the paper gives none); a_uv = P_dot / (rho dV).
struct UvArgs {
    const float* nph;
    const float* uph;
    const float* xion;
    const float* rho;
    const int4* geo;
    const int32_t* leaf_node;
    const int32_t* inv_perm;
    float *a, *f;
    int64_t n;
    double box;
};

__global__ void k_uv_radpressure(UvArgs r) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= r.n) return;
    constexpr double kSigmaD = 1.5e-21, kSigmaH = 6.3e-18, kAlphaB = 2.5e-13;
    constexpr double kEoverC = 18.0 * 1.602176634e-12 / kLightC;
    const int lvl = r.geo[r.leaf_node[r.inv_perm[k]]].z >> 24;
    const double dx = ldexp(r.box, -lvl);
    const double dV = (dx * dx) * dx;
    const double rho = (double)r.rho[k];
    const double nh = kHydrogenFraction * rho / kHydrogenMass;
    const double x = r.xion ? (double)r.xion[k] : 1.0;
    const double N = (double)r.nph[k];
    const double n0 = (1.0 - x) * nh, np = x * nh;
    const double rate = kSigmaD * nh * N + kSigmaH * n0 * N + kAlphaB * np * np;
    for (int ax = 0; ax < 3; ++ax) {
        const double pd = kEoverC * rate * (double)r.uph[3 * k + ax] * dV;
        if (r.f) r.f[3 * k + ax] = (float)pd;
        if (r.a) r.a[3 * k + ax] = (float)(pd / (rho * dV));
    }
}

struct DustArgs {
    const int* skip;
    const float* rho;
    const float* tgas;
    const float* heat;
    const float* J;
    const float* kin;
    float* Td;
    int64_t n;
    int model;
    double kappa0, xi;
    unsigned* err;  // kErrInput for a negative or non-finite gas temperature or heating rate
};

__device__ inline double kappa_of(const DustArgs& d, int64_t k, double T) {
    if (d.kin) return (double)d.kin[k];
    if (d.model == 0) return d.kappa0;
    const double Tc = T < 150.0 ? T : 150.0;
    return 1.0e-3 * (Tc * Tc);
}

// Per-cell constants of G(T) that do not depend on T_d, kept in the evaluation order
// of the full expression so that G is rounded exactly as if written out:
// gd = ((((3.8e-33 sqrt(Tg)) (Tg - T)) (1 - 0.8 e^(-75/Tg))) n_H^2) (xi / 0.01)
struct Cell {
    double c1;   // 3.8e-33 sqrt(Tg)
    double c2;   // 1 - 0.8 exp(-75 / Tg)
    double nH2;  // n_H^2
    double Tg, rho, J, H;
};

// G(T) = Gamma_dust-gas + heat + rho kappa(T) (4 pi J - 4 sigma T^4)
__device__ inline double balance(const DustArgs& d, int64_t k, const Cell& c, double T) {
    const double kap = kappa_of(d, k, T);
    const double gd = c.c1 * (c.Tg - T) * c.c2 * c.nH2 * (d.xi / 0.01);
    const double T4 = (T * T) * (T * T);
    return gd + c.H + c.rho * kap * (4.0 * kPi * c.J - 4.0 * kSigmaSB * T4);
}

// The reference procedure: 60 bisections in ln T on [floor, hi]; the root to FP64
// precision (used where the fast path below cannot vouch for its bracket).
__device__ double bisect64(const DustArgs& d, int64_t k, const Cell& c, double lo, double hi) {
    for (int it = 0; it < 60; ++it) {
        const double mid = sqrt(lo * hi);
        if (balance(d, k, c, mid) > 0.0) lo = mid;
        else hi = mid;
    }
    return sqrt(lo * hi);
}

// The same root, found in two stages so that the GB300's slow FP64 pipe does little work:
// bisection in ln T in FP32 on G scaled by 1/M (M bounds every term of G on [floor, hi]),
// until the bracket is two adjacent floats; then FP64 checks that G changes sign across
// it (stepping by single floats when the FP32 signs misled it) and picks the float nearest
// the root from the sign of G at the bracket's midpoint, i.e. the root rounded to FP32.
__device__ double root_two_stage(const DustArgs& d, int64_t k, const Cell& c, double hi64) {
    const double b = c.c1 * c.c2 * c.nH2 * (d.xi / 0.01);  // G_dust-gas = b (T_gas - T)
    const double M = fabs(c.H) + fabs(b) * (c.Tg + hi64) +
                     c.rho * kappa_of(d, k, hi64) * (4.0 * kPi * c.J + 4.0 * kSigmaSB * ((hi64 * hi64) * (hi64 * hi64)));
    if (!(M > 0.0) || !(M < 1e300)) return bisect64(d, k, c, kDustFloorK, hi64);
    const double sc = 1.0 / M;
    const float Hs = (float)(c.H * sc), bs = (float)(b * sc), rs = (float)(c.rho * sc), Tg = (float)c.Tg;
    const float J4 = (float)(4.0 * kPi * c.J), s4 = (float)(4.0 * kSigmaSB);
    const float kc = d.kin ? d.kin[k] : (float)d.kappa0;
    float lo = (float)kDustFloorK, hi = (float)hi64;
    for (int it = 0; it < 96; ++it) {
        float mid = sqrtf(lo) * sqrtf(hi);
        // a few units apart the rounded geometric mean can fall on an end point: the
        // arithmetic mean of the two floats then still splits the bracket
        if (!(mid > lo && mid < hi)) mid = 0.5f * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        const float Tc = fminf(mid, 150.0f);
        const float kap = (d.kin || d.model == 0) ? kc : 1.0e-3f * (Tc * Tc);
        const float T4 = (mid * mid) * (mid * mid);
        const float g = Hs + bs * (Tg - mid) + rs * kap * (J4 - s4 * T4);
        if (g > 0.0f) lo = mid;
        else hi = mid;
    }
    bool ok = false;
    for (int it = 0; it < 8; ++it) {
        if (!(balance(d, k, c, (double)lo) > 0.0)) {  // root below lo
            hi = lo;
            lo = nextafterf(lo, 0.0f);
            continue;
        }
        if (balance(d, k, c, (double)hi) > 0.0) {  // root above hi
            lo = hi;
            hi = nextafterf(hi, 3.0e38f);
            continue;
        }
        ok = true;
        break;
    }
    if (!ok || nextafterf(lo, 3.0e38f) != hi) return bisect64(d, k, c, kDustFloorK, hi64);
    const double m = 0.5 * ((double)lo + (double)hi);
    return balance(d, k, c, m) > 0.0 ? (double)hi : (double)lo;
}

// root by bracketing from the 2.7 K floor (as the reference procedure), then the two-stage
// search for the FP32 result
__global__ void k_dust(DustArgs d) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= d.n || (d.skip && *d.skip)) return;
    Cell c;
    c.rho = (double)d.rho[k];
    c.Tg = (double)d.tgas[k];
    c.J = (double)d.J[k];
    c.H = d.heat ? (double)d.heat[k] : 0.0;
    if (!(c.Tg >= 0.0 && c.Tg <= 3.4e38) || !(c.H >= -3.4e38 && c.H <= 3.4e38)) atomicOr(d.err, kErrInput);
    c.c1 = 3.8e-33 * sqrt(c.Tg);
    c.c2 = 1.0 - 0.8 * exp(-75.0 / c.Tg);
    const double nH = kHydrogenFraction * c.rho / kHydrogenMass;
    c.nH2 = nH * nH;
    double T;
    if (balance(d, k, c, kDustFloorK) <= 0.0) {
        T = kDustFloorK;
    } else {
        const double TJ = sqrt(sqrt(kPi * (c.J > 0.0 ? c.J : 0.0) / kSigmaSB));
        double hi = c.Tg > TJ ? c.Tg : TJ;
        if (hi < kDustFloorK) hi = kDustFloorK;
        for (int it = 0; it < 64 && balance(d, k, c, hi) > 0.0; ++it) hi *= 2.0;
        T = root_two_stage(d, k, c, hi);
    }
    d.Td[k] = (float)T;
}

}  // namespace

treeray_status launch_radpressure(treeray_ctx* c, const float* J, const double* F, float* u, float* a,
                                  float* f, float* p, cudaStream_t s) {
    RpArgs r{J, F, c->tree.kap, c->tree.tau, c->tree.psrc, c->tree.rho, c->tree.geo, c->tree.leaf_node,
             c->tree.inv_perm, u, a, f, p, c->nleaves, c->box};
    k_radpressure<<<(int)((c->nleaves + 255) / 256), 256, 0, s>>>(r);
    c->launches += 1;
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}

treeray_status launch_uv_radpressure(treeray_ctx* c, const float* nph, const float* uph, const float* xion,
                                     float* a, float* f, cudaStream_t s) {
    UvArgs r{nph, uph, xion, c->tree.rho, c->tree.geo, c->tree.leaf_node, c->tree.inv_perm, a, f, c->nleaves, c->box};
    k_uv_radpressure<<<(int)((c->nleaves + 255) / 256), 256, 0, s>>>(r);
    c->launches += 1;
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}

treeray_status launch_dust(treeray_ctx* c, const float* Tgas, const float* heat, const float* J, float* Td,
                           cudaStream_t s) {
    return launch_dust_skip(c, Tgas, heat, J, Td, nullptr, s);
}

treeray_status launch_dust_skip(treeray_ctx* c, const float* Tgas, const float* heat, const float* J,
                                float* Td, const int* skip, cudaStream_t s) {
    DustArgs d{skip, c->tree.rho, Tgas, heat, J, c->kin_given ? c->tree.kin : nullptr, Td, c->nleaves,
               c->p.kappa_model, c->p.kappa0, c->p.dust_to_gas, c->dt.err};
    k_dust<<<(int)((c->nleaves + 127) / 128), 128, 0, s>>>(d);
    c->launches += 1;
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}

namespace {
// Warm-start features of every leaf (caller order), as 6 floats:
//   log10 rho, log10 T_gas, log10(mean ray optical depth + 1e-6), log10(ionising flux + 1),
//   log10(smallest ray optical depth + 1e-6), log10(J of the same evaluation + 1e-30)
struct FeatArgs {
    const float* rho;
    const float* tgas;
    const float* phi;
    const float* tau_mean;
    const float* tau_min;
    const float* J;
    int64_t n;
    float* X;
};

__global__ void k_features(FeatArgs f) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= f.n) return;
    float* x = f.X + 6 * k;
    x[0] = log10f(f.rho[k]);
    x[1] = log10f(f.tgas[k]);
    x[2] = log10f(f.tau_mean[k] + 1e-6f);
    x[3] = log10f((f.phi ? f.phi[k] : 0.0f) + 1.0f);
    x[4] = log10f(f.tau_min[k] + 1e-6f);
    x[5] = log10f(f.J[k] + 1e-30f);
}

// Largest relative change max_k |T_new - T| / T of one fixed-point iteration (as the
// bits of a non-negative float, whose integer order is the float order); T <- T_new.
__global__ void k_fp_delta(const float* Tnew, float* T, int64_t n, int* flags) {
    if (flags[0]) return;
    float m = 0.0f;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float t0 = T[k], t1 = Tnew[k];
        m = fmaxf(m, fabsf(t1 - t0) / t0);
        T[k] = t1;
    }
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned*>(flags + 2), __float_as_uint(m));
}

// count the iteration; converged (1) when the largest change is below tol, out of
// iterations (2) at max_iter
__global__ void k_fp_check(int* flags, float tol, int max_iter) {
    if (flags[0]) return;
    flags[1] += 1;
    const float m = __uint_as_float((unsigned)flags[2]);
    if (m < tol) flags[0] = 1;
    else if (flags[1] >= max_iter) flags[0] = 2;
    flags[2] = 0;
}
}  // namespace

treeray_status launch_features(treeray_ctx* c, const float* Tgas, const float* phi, const float* tau_mean,
                               const float* tau_min, const float* J, float* X, cudaStream_t s) {
    FeatArgs f{c->tree.rho, Tgas, phi, tau_mean, tau_min, J, c->nleaves, X};
    k_features<<<(int)((c->nleaves + 255) / 256), 256, 0, s>>>(f);
    c->launches += 1;
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}

treeray_status launch_fp_update(treeray_ctx* c, const float* Tnew, float* Td, double tol, int max_iter,
                                cudaStream_t s) {
    int sms = 0;
    TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    int64_t blocks = std::min<int64_t>((c->nleaves + 255) / 256, (int64_t)sms * 8);
    if (blocks < 1) blocks = 1;
    k_fp_delta<<<(int)blocks, 256, 0, s>>>(Tnew, Td, c->nleaves, c->fp_flags);
    k_fp_check<<<1, 1, 0, s>>>(c->fp_flags, (float)tol, max_iter);
    c->launches += 2;
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}

}  // namespace tr
