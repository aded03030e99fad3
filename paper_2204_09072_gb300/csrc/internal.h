// Internal declarations of the treeray CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/treeray.h"

namespace tr {

// physical constants, CGS
constexpr double kPi = 3.14159265358979323846;
constexpr double kSigmaSB = 5.670374419e-5;
constexpr double kLightC = 2.99792458e10;
constexpr double kHydrogenMass = 1.6726e-24;
constexpr double kHydrogenFraction = 0.7;
constexpr double kDustFloorK = 2.7;

constexpr int kMaxLevel = 19;     // octree levels below the root
constexpr int kMaxBins = 64;
constexpr int kMaxStars = 4096;
constexpr int kMaxOrientations = 64;

// device error word bits
enum : unsigned {
    kErrStack = 1u,       // walk stack overflow
    kErrAlphaKey = 2u,    // angular-kernel key outside the table
    kErrOctree = 4u,      // the leaves do not form a complete octree
    kErrTarget = 8u,      // target index out of range
    kErrInput = 16u,      // a density, temperature or opacity input is negative or not finite
};

void set_error(const std::string& msg);

// An NVTX range named after the ABI call for the scope of one call (a no-op unless a
// profiler such as Nsight Systems or Nsight Compute with --nvtx listens).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Host-built tables (FP64 on the host, fixed per context and grid shape).
struct HostTables {
    int npix = 0, nside = 0, s = 8;
    std::vector<float> nhat;          // [orientations][npix][3] ray directions (pixel centres)
    int D = 0;                        // alpha keys cover |K_a| <= D
    std::vector<int32_t> alpha_off;   // [orientations][(2D+1)^3 + 1]
    std::vector<uint32_t> alpha_ent;  // pixel | count << 16
};

int healpix_nside(int npix);
int healpix_ang2pix(int nside, double x, double y, double z);
void healpix_pix2vec(int nside, int pix, double* v);
void alpha_counts(int npix, int s, const int64_t* K, int32_t* counts, const double* rot = nullptr);
// Build the alpha table for the keys the walk can reach on this grid shape, one per
// orientation in rot (k row-major rotations; none: the unturned grid). False when the
// entries outgrow 32-bit offsets.
bool build_alpha_table(HostTables& t, double theta, int lmax, bool amr, bool col, const std::vector<double>& rot);
// Evaluation radii R_i (half-cells of the finest level) for a target of edge Et.
void radii(int nbins, int lmax, int periodic, int spacing, int64_t Et, double* R);

struct DeviceTree {
    // per node (breadth first)
    int4* geo = nullptr;           // cx, cy, cz | level << 24, child0 or -1 - sorted leaf
    float4* thin = nullptr;        // Lt, At, colx, coly  (internal units)
    float4* thick = nullptr;       // colz, LVk, Ak, Vk   (internal units)
    double* mom = nullptr;         // [11][nn] FP64 moments (SoA)
    uint64_t* prefix = nullptr;    // Morton prefix at the node's level
    // per leaf
    uint64_t* keys = nullptr;      // sorted keys (level << 3 lmax | Morton)
    int32_t* perm = nullptr;       // sorted leaf -> caller index
    int32_t* inv_perm = nullptr;   // caller index -> sorted leaf
    int32_t* leaf_node = nullptr;  // sorted leaf -> node id
    double* kap = nullptr;         // caller order
    double* tau = nullptr;
    double* jsrc = nullptr;
    double* psrc = nullptr;
    int32_t* thickflag = nullptr;
    float* rho = nullptr;          // caller order copy
    float* kin = nullptr;          // caller-given opacity copy (or null)
    // scratch for the build
    uint64_t* keys_alt = nullptr;
    int32_t* vals_alt = nullptr;
    uint32_t* hist = nullptr;
    double* stars = nullptr;       // [cap_stars][4] x, y, z, L
    int4* blocks = nullptr;        // AMR block table
    int* levels = nullptr;         // [2][kMaxLevel + 1] leaf ranges per level
    int64_t cap_leaves = 0, cap_nodes = 0, cap_hist = 0, cap_stars = 0, cap_blocks = 0;
};

struct DeviceTables {
    float* nhat = nullptr;
    int32_t* alpha_off = nullptr;
    int2* alpha_pair = nullptr;     // [orientations][(2D+1)^3] (first entry, end) of each key
    uint32_t* alpha_ent = nullptr;
    int64_t* bin_thr = nullptr;     // [lmax+1][nbins] ceil(R_i^2), i>=1 used
    longlong2* bin_thr2 = nullptr;  // [lmax+1][nbins] (thr[i], thr[i+1]), thr[nbins] = INT64_MAX
    float* R2 = nullptr;            // [lmax+1][nbins] R_i^2 (half-cells^2)
    float* Rh = nullptr;            // [lmax+1][nbins] R_i (half-cells)
    double* Rd = nullptr;           // [lmax+1][nbins] R_i in FP64 (decisions at the COL)
    float2* lvlp = nullptr;         // [lmax+1] 1 / R_0^2 and 0.5 / log2(g) (segment guess)
    int64_t* open_max = nullptr;    // [lmax+1] largest d^2 at which a node of that level opens
    int64_t* str_lo = nullptr;      // [lmax+1 target][lmax+1 node][nbins] straddle thresholds
    int64_t* str_hi = nullptr;
    double* scal = nullptr;         // [0] luminosity scale (erg/s, power of two)
    unsigned* err = nullptr;        // device error word
    unsigned long long* queue = nullptr;  // work counter of the persistent kernels
};

}  // namespace tr

struct treeray_ctx {
    treeray_params p{};
    int device = 0;
    tr::HostTables ht;
    tr::DeviceTables dt;
    tr::DeviceTree tree;
    // current grid
    bool built = false;
    bool amr = false;
    int lmax = -1;
    double box = 0, u = 0;  // box edge and half-cell of the finest level (cm)
    int64_t nleaves = 0, nnodes = 0;
    int level_off[tr::kMaxLevel + 2] = {0};
    int level_cnt[tr::kMaxLevel + 2] = {0};
    bool has_thick = false;
    bool kin_given = false;
    bool force_thick = false;  // fixed point: thin/thick classes may change between refreshes
    int grid_n = 0, n_stars = 0;
    // fixed-point scratch
    float* fp_Tnew = nullptr;
    float* fp_J = nullptr;
    double* fp_F = nullptr;
    int* fp_flags = nullptr;       // [0] done (1 converged, 2 out of iterations), [1] iterations, [2] max change bits
    int64_t fp_cap = 0;
    cudaStream_t fp_stream = nullptr;
    cudaEvent_t fp_ev[2] = {nullptr, nullptr};
    int* stack_scr = nullptr;    // evaluate: team stacks (global scratch, grow-only)
    size_t stack_scr_bytes = 0;
    float* gtile = nullptr;      // evaluate at 768 rays: the teams' tiles (global scratch, grow-only)
    size_t gtile_bytes = 0;
    // several HEALPix orientations (Sec. 7.6)
    std::vector<double> rot;     // [k][9] row-major rotations; empty: the single unturned ray set
    uint8_t* orient = nullptr;   // device [orient_n]: orientation of each leaf (caller order)
    int64_t orient_n = 0;        // leaves the map was made for
    bool orient_user = false;    // the map came from the caller (else leaf mod k)
    int64_t launches = 0;  // kernels launched by this context
    int wpt = 4;           // warps per target team of the evaluate kernel (autotuned)
    int occ_pct = 100;     // evaluate: resident teams per SM launched, % of the maximum (autotuned)
    int stack_limit = 0;   // test hook: cap on the walk stack's entries (0: the full stack)
    int alloc_fail_at = 0; // test hook: the n-th device allocation from now fails (0: none)
    int alloc_count = 0;
    // table cache key
    int tab_lmax = -1;
    bool tab_amr = false;
    int64_t tab_D = -1;
};

// kernels entry points (defined in the .cu files)
namespace tr {
// Device allocation of a context's buffers (cudaMalloc), or the failure that
// treeray_inject_alloc_failure arranged; on failure *p is null and TREERAY_ENOMEM returned.
treeray_status dev_alloc(treeray_ctx* c, void** p, size_t bytes);
// Team-stack scratch of the evaluate kernel large enough for any team size on a tree of
// `lmax` levels below the root; never allocates while `s` is being captured.
treeray_status reserve_eval_stacks(treeray_ctx* c, int lmax, cudaStream_t s);
treeray_status reserve_team_tiles(treeray_ctx* c, int64_t n, cudaStream_t s);
treeray_status reserve_team_tiles_kind(treeray_ctx* c, int64_t n, bool thick, cudaStream_t s);
// Apply the autotuner's choice cached for a tree of this context's shape, if any.
void apply_cached_launch_choice(treeray_ctx* c);
treeray_status build_tree(treeray_ctx* c, const treeray_grid* g, const float* rho, const float* Td,
                          const float* kappa, int n_stars, const double* star_pos,
                          const double* star_lum, cudaStream_t s);
treeray_status launch_evaluate(treeray_ctx* c, const int32_t* targets, int64_t n, float* J,
                               double* F, cudaStream_t s);
treeray_status launch_accepted(treeray_ctx* c, const int32_t* targets, int64_t n, int32_t cap,
                               int32_t* counts, int32_t* ids, cudaStream_t s);
treeray_status launch_walk_stats(treeray_ctx* c, const int32_t* targets, int64_t n, int64_t* totals,
                                 cudaStream_t s);
treeray_status launch_uv_radpressure(treeray_ctx* c, const float* nph, const float* uph, const float* xion,
                                     float* a, float* f, cudaStream_t s);
treeray_status launch_radpressure(treeray_ctx* c, const float* J, const double* F, float* u,
                                  float* a, float* f, float* p, cudaStream_t s);
treeray_status launch_dust(treeray_ctx* c, const float* Tgas, const float* heat, const float* J,
                           float* Td, cudaStream_t s);
treeray_status upload_tables(treeray_ctx* c, cudaStream_t s);
treeray_status refresh_tree(treeray_ctx* c, const float* Td, const int* skip, cudaStream_t s);
treeray_status launch_evaluate_tau(treeray_ctx* c, float* J, double* F, float* tau_mean, float* tau_min,
                                   cudaStream_t s);
treeray_status launch_features(treeray_ctx* c, const float* Tgas, const float* phi, const float* tau_mean,
                               const float* tau_min, const float* J, float* X, cudaStream_t s);
treeray_status launch_evaluate_skip(treeray_ctx* c, float* J, double* F, const int* skip, cudaStream_t s);
treeray_status launch_dust_skip(treeray_ctx* c, const float* Tgas, const float* heat, const float* J,
                                float* Td, const int* skip, cudaStream_t s);
treeray_status launch_fp_update(treeray_ctx* c, const float* Tnew, float* Td, double tol, int max_iter,
                                cudaStream_t s);
void free_tree(tr::DeviceTree& t);
void free_tables(tr::DeviceTables& t);
}  // namespace tr

#define TR_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            tr::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
            return e_ == cudaErrorMemoryAllocation ? TREERAY_ENOMEM : TREERAY_ECUDA;        \
        }                                                                                  \
    } while (0)
