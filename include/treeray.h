/*
 * treeray.h - C ABI of the GB300 (sm_103a) TreeRay/RadPressure hot path.
 *
 * Backwards ray tracing of infrared radiation from diffuse sources on an
 * octree, after Klepitko, Walch, Wuensch, Seifried, Dinnbier & Haid (MNRAS 2023),
 * "Tree-based solvers for adaptive mesh refinement code FLASH - III".
 * Every cell and every star particle emits; for each target cell N_pix HEALPix
 * rays are cast, the tree is walked under an opening criterion, accepted nodes
 * are deposited into the radial segments of the rays they cover, each ray is
 * integrated from the inside out and the rays are reduced to J, F, u and the
 * radiation-pressure terms.
 *
 * Conventions
 *  - Units are CGS. Grids are cubic; positions are in [0, box)^3.
 *  - Leaves are given in the caller's order: x fastest for a uniform n^3 grid,
 *    block-major then x fastest inside each 8^3 block for AMR grids. Every
 *    per-leaf input and output array uses that order.
 *  - "device" pointers are CUDA global-memory pointers on the context's device;
 *    "host" pointers are ordinary host memory. The caller owns every array it
 *    passes; the context owns the tree, the tables and its scratch memory.
 *  - Calls that take a cudaStream_t enqueue their work on that stream and return
 *    before it finishes, unless stated otherwise. Errors found by a kernel are
 *    recorded in a device error word and reported by treeray_check().
 *  - Functions return a treeray_status; treeray_last_error() gives the message.
 *    No function aborts the process.
 *  - A context is bound to the device that was current at treeray_create(); call
 *    every function with that device current. Contexts are not thread-safe.
 */
#ifndef TREERAY_H
#define TREERAY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct treeray_ctx* treeray_t;
typedef struct CUstream_st* treeray_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    TREERAY_OK = 0,
    TREERAY_EINVAL = 1,     /* bad argument or unsupported size */
    TREERAY_ENOMEM = 2,     /* device or host allocation failed */
    TREERAY_ECUDA = 3,      /* a CUDA runtime call failed */
    TREERAY_ENOTBUILT = 4,  /* evaluate/radpressure/dust before a successful build */
    TREERAY_ETIMEOUT = 5,   /* a bounded device loop ran out (stack overflow, table miss) */
    TREERAY_ENOCONV = 6     /* the dust-temperature fixed point did not converge */
} treeray_status;

/*
 * Method parameters.
 *  npix            HEALPix rays per target, 12 * nside^2 with nside in {1, 2, 4}
 *                  (Sec. 4.2 "Ray mapping").
 *  nbins           radial evaluation points per ray, 1..64. Evaluation point i sits
 *                  at R_i = R_0 (R_max/R_0)^(i/nbins), R_0 = half the target cell,
 *                  R_max = sqrt(3) box; segment i is [R_i, R_(i+1)) and segment 0
 *                  also holds [0, R_0) (Sec. 4.2, Fig. "ray bin").
 *  theta           opening angle theta_lim: a node of edge E at distance d from the
 *                  target (centre to centre) is opened iff E^2 >= theta^2 d^2, or if
 *                  it contains the target; leaves are always accepted (Sec. 4). In
 *                  (0, 2]; a negative value selects the angle matched to the ray size,
 *                  sqrt(4 pi / npix) (Sec. 7.6: more rays open nodes further).
 *  kappa_model     0: grey kappa0 per gram of gas; 1: Planck mean
 *                  0.1 cm^2/g (T/10 K)^2 capped at 150 K (Sec. 2).
 *  kappa0          grey opacity, cm^2/g (kappa_model 0).
 *  dust_to_gas     xi; enters only the gas-dust coupling of the dust temperature.
 *  dust_emission   1: dust emits (eqs. lthinbnode, lthickbnode); 0: only stars emit
 *                  (the point-source benchmark, Sec. 5.1).
 *  kappa_ext_scale multiplies the extinction areas A~ (1 = the method; 0 = test switch).
 *  alpha_s         sub-cube samples per axis of the angular kernel, a multiple of 4
 *                  (8 is the default, 512 samples per node position).
 *  periodic        bit a (x = 1, y = 2, z = 4) set: axis a is periodic. Every node then
 *                  enters at its closest periodic copy (Sec. 4.2, periodic boundaries); a
 *                  node exactly half a box away on such an axis has two closest copies and
 *                  enters at both, each with weight 1/2. R_max becomes the largest
 *                  closest-copy distance, sqrt of the sum over axes of (box/2)^2 on
 *                  periodic and box^2 on isolated axes. 0 (all isolated) is the default.
 *  bin_spacing     0: geometric radii as above (the default); 1: radii growing
 *                  quadratically, R_i = R_0 + (R_max - R_0) (i / nbins)^2 (Sec. 4.2, "grows
 *                  quadratically").
 *  col_mapping     0: accepted nodes are mapped at their geometric centre (the default);
 *                  1: at their centre of luminosity (Sec. 7.6, nodes shifted towards their
 *                  centre of emission): for a node whose COL is off centre, the segment,
 *                  the straddled boundaries and the angular key come from the COL offset
 *                  in FP32 (p = centre offset + COL offset, p^2 against the integer
 *                  thresholds, key 2 floor(4 p / E) + 1 per axis).
 */
typedef struct {
    int npix;
    int nbins;
    double theta;
    int kappa_model;
    double kappa0;
    double dust_to_gas;
    int dust_emission;
    double kappa_ext_scale;
    int alpha_s;
    int periodic;
    int bin_spacing;
    int col_mapping;
} treeray_params;

/*
 * Grid description.
 *  Uniform: n > 0 is the cells per axis (a power of two, 1..2^10); n_blocks = 0.
 *  AMR:     n = 0; n_blocks > 0 blocks of 8^3 cells; blocks is a HOST array of
 *           4 ints per block (bi, bj, bk, l): the block's cells sit at octree level l
 *           (root = level 0, cell edge box / 2^l) with integer coordinates
 *           8 (bi, bj, bk) + (x, y, z). The blocks must tile the box and form a
 *           complete octree (every refined region split into 8).
 *  box: box edge in cm.
 */
typedef struct {
    int n;
    int n_blocks;
    const int32_t* blocks;
    double box;
} treeray_grid;

/* Create a context on the current device: validates params and builds the
 * HEALPix ray directions on the host. Returns TREERAY_EINVAL for bad params. */
treeray_status treeray_create(const treeray_params* params, treeray_t* out);

/* Destroy a context and free everything it owns. NULL is allowed. */
treeray_status treeray_destroy(treeray_t ctx);

/*
 * Several HEALPix orientations (Sec. 7.6: with one orientation for every target the rays
 * imprint a ray-like pattern on the radiation field; turning the ray set from target to
 * target breaks it up, at the price of one angular-kernel table per orientation).
 *  k       number of orientations, 1..64; 0 goes back to the single unturned ray set
 *          (the default).
 *  rot     HOST double[9 k], row-major 3x3 rotations R_o (orthonormal to 1e-9,
 *          determinant +1; copied). Ray h of orientation o points along R_o n_h, n_h the
 *          HEALPix pixel centre; a direction v lies in ray h of orientation o when
 *          R_o^T v lies in pixel h. The angular kernel of orientation o counts each of
 *          a node's alpha_s^3 sample directions v in the pixel of R_o^T v, computed in
 *          FP64 as (R^T v)_a = R_0a v_x + R_1a v_y + R_2a v_z.
 *  orient  DEVICE uint8[N] (N leaves of the built grid, caller order; copied): the
 *          orientation of each target, every value < k. NULL: leaf l uses l mod k. A
 *          caller map needs a built tree, and a later build with another leaf count
 *          replaces it by l mod k.
 * The tables are rebuilt at once (host FP64, about 0.1-0.2 s per orientation at
 * theta = 0.5) when a tree is built, else at the next build. Synchronises the device.
 * EINVAL: k out of range, rot missing or not a rotation, a map value >= k, a map
 * without k; ENOTBUILT: a map before any build; ENOMEM: the tables of all orientations
 * outgrow 2^31 entries or device memory.
 */
treeray_status treeray_set_orientations(treeray_t ctx, int k, const double* rot, const uint8_t* orient);

/*
 * Tree build (Sec. 4.1 and App. A): leaf quantities, Morton sort, node structure,
 * node moments and the centre of luminosity, plus the angular-kernel table.
 *  rho, Td         device float[N]: gas density (g/cm^3), dust temperature (K).
 *  kappa           device float[N] opacity (cm^2/g) or NULL to use the params' model.
 *  n_stars         number of point sources (0..4096).
 *  star_pos        host double[3 n_stars] positions (cm); star_lum host double[n_stars]
 *                  non-ionising luminosity L_src,IR (erg/s). A star heats the leaf whose
 *                  half-open cell contains its position.
 * Per leaf (Sec. 4.1.1): tau_b = rho kappa dx; thin iff tau_b < 1; thin: L = 4 sigma
 * rho kappa T^4 dV, A~ = rho kappa dV; thick: L_ = (sigma/pi) T^4, A~; S = L_src
 * e^(-tau_b/2); J_src = (1 - e^(-tau_b/2)) L_src / dx^2 (eq. jsrc);
 * P_src = (1 - e^(-tau_b/2)) L_src / (c dx^2) (eq. psrc).
 * The call synchronizes the stream once (to size the tree) and returns after the
 * build is enqueued. Inputs may be freed after the stream has finished. It also reserves
 * the evaluation scratch for up to N targets (team stacks, and the teams' ray tiles in
 * global memory: at most 96 MB), so that evaluations can be captured in a CUDA graph.
 */
treeray_status treeray_build(treeray_t ctx, const treeray_grid* grid, const float* rho,
                             const float* Td, const float* kappa, int n_stars,
                             const double* star_pos, const double* star_lum,
                             treeray_stream_t stream);

/*
 * Ray evaluation (Secs. 4.2-4.4): walk, ray mapping with the angular kernel alpha and
 * radial kernel beta = R_i^2 / r^2, segment merge, ray integration and finalization
 * F = sum_h -F^h n^h, J = (1/4pi) sum_h F^h + J_src.
 *  targets   device int32[n] caller leaf indices, or NULL for every leaf (then
 *            n must equal the leaf count and row k of the outputs is leaf k). n = 0 is
 *            an empty list: nothing is launched or written.
 *  J         device float[n], mean intensity (erg/s/cm^2/sr).
 *  F         device double[3n], flux vector xyz interleaved (erg/s/cm^2).
 * A target list longer than the leaf count may need more scratch than the build
 * reserved: outside a stream capture it is grown, inside one the call returns
 * TREERAY_EINVAL.
 */
treeray_status treeray_evaluate(treeray_t ctx, const int32_t* targets, int64_t n, float* J,
                                double* F, treeray_stream_t stream);

/*
 * Radiation energy density and pressure (Sec. 4.5) for every leaf (caller order):
 *  u = 4 pi J / c; P_dot = (F/c) kappa rho (1 - e^-tau)/tau dV (the tau factor is 1 for
 *  tau < 1e-4); a_rp = P_dot / (rho dV); force = P_dot; p_src from the build.
 *  J device float[N], F device double[3N]; outputs device float: u[N], a_rp[3N],
 *  force[3N], p_src[N]. Any output may be NULL.
 */
treeray_status treeray_radpressure(treeray_t ctx, const float* J, const double* F, float* u,
                                   float* a_rp, float* force, float* p_src,
                                   treeray_stream_t stream);

/*
 * Radiation pressure of the ionising (UV) radiation on dust, neutral and ionised hydrogen
 * (Sec. 4.5 and App. C), for every leaf (caller order), from a given ionising field (the
 * transfer of ionising radiation itself is a separate module in the paper):
 *  P_dot = (E/c) [sigma_d n N + sigma_H (1 - x) n N + alpha_B (x n)^2] u dV,
 *  a_uv = P_dot / (rho dV), force_uv = P_dot,
 * with n = 0.7 rho / m_H hydrogen nuclei per cm^3, E = 18 eV per photon, sigma_d =
 * 1.5e-21 cm^2 per H, alpha_B = 2.5e-13 cm^3/s (the paper's values) and sigma_H =
 * 6.3e-18 cm^2 (the Lyman-edge cross-section; the paper gives none).
 *  nph     device float[N], ionising photons per s and cm^2 arriving at the cell.
 *  uph     device float[3N], unit direction of that photon flux, xyz interleaved.
 *  x_ion   device float[N], ionised fraction of hydrogen, or NULL (fully ionised).
 *  a_uv, force_uv: device float[3N] outputs (cm/s^2, dyn); either may be NULL.
 * Needs a built tree (density and cell sizes); TREERAY_EINVAL if nph or uph is NULL.
 */
treeray_status treeray_uv_radpressure(treeray_t ctx, const float* nph, const float* uph,
                                      const float* x_ion, float* a_uv, float* force_uv,
                                      treeray_stream_t stream);

/*
 * Equilibrium dust temperature (Sec. 4.6, App. D) per leaf (caller order): the root of
 *  Gamma_dust-gas + heat_extra + rho kappa(T_d) (4 pi J - 4 sigma T_d^4) = 0,
 *  Gamma_dust-gas = 3.8e-33 sqrt(T) (T - T_d)(1 - 0.8 e^(-75/T)) n_H^2 (xi/0.01),
 *  n_H = 0.7 rho / m_H, floor 2.7 K. The result is the FP32 value of the root that
 *  bracketing and 60 bisections in ln T give in FP64 (reached by FP32 bisection with
 *  FP64 sign checks of G around the final float).
 *  Tgas device float[N]; heat_extra device float[N] (erg/s/cm^3) or NULL; J device
 *  float[N]; Td device float[N] output. rho (and kappa if given) from the build.
 */
treeray_status treeray_dust_temperature(treeray_t ctx, const float* Tgas, const float* heat_extra,
                                        const float* J, float* Td, treeray_stream_t stream);

/*
 * New dust temperatures on the grid of the last treeray_build (same densities, opacity
 * input and stars): recompute the leaf quantities, node moments and centres of
 * luminosity (Sec. 4.1) without rebuilding keys or structure. Td device float[N].
 * Asynchronous and free of host synchronisation (it can be captured in a CUDA graph).
 */
treeray_status treeray_refresh(treeray_t ctx, const float* Td, treeray_stream_t stream);

/*
 * Dust-temperature / IR-field fixed point on the grid of the last treeray_build: repeat
 *   T_d -> tree moments -> J (treeray_evaluate) -> T_new (treeray_dust_temperature)
 * until max_k |T_new - T_d| / T_d < tol (the paper couples T_d and the IR field with a
 * lag of one hydro step, Sec. 4.6; converging the coupling is the fixed point's job).
 *  Tgas device float[N]; heat_extra device float[N] or NULL; Td device float[N]: the
 *  initial guess on entry, the converged temperatures on return.
 *  max_iter   iteration limit; tol relative tolerance (e.g. 1e-4).
 *  unroll     0: one host round trip per iteration; k > 0: the loop runs as a CUDA
 *             graph of k iterations replayed until a device flag reports convergence
 *             (iterations past convergence do nothing).
 *  iters      host int: iterations performed (the converging one included).
 * Synchronous: returns when done. TREERAY_ENOCONV when max_iter is reached first.
 */
treeray_status treeray_fixed_point(treeray_t ctx, const float* Tgas, const float* heat_extra,
                                   float* Td, int max_iter, double tol, int unroll, int* iters,
                                   treeray_stream_t stream);

/*
 * Warps per target for the evaluate kernel, chosen by timing (autotuner): the evaluate
 * kernel runs a team of 2, 3, 4 or 8 warps per target sharing one walk stack and one ray
 * tile (3 only for trees without thick material below 768 rays; elsewhere a request for 3
 * runs teams of 4); each choice is launched twice on
 * n_sample targets of the current tree (a fixed stride permutation of the leaves) and the
 * second launch is timed. The fastest choice is kept by the context. best_wpt (host int)
 * and ms (host float[4], times for 2, 3, 4, 8; -1 for a choice not tried) may be NULL.
 * Synchronous.
 */
treeray_status treeray_autotune(treeray_t ctx, int64_t n_sample, int* best_wpt, float* ms,
                                treeray_stream_t stream);

/*
 * The autotuner over both result-neutral launch choices of the evaluate kernel (no
 * counterpart in the paper; the method's results do not depend on them): warps per target
 * team as treeray_autotune does, then, for the fastest team size, the resident teams per SM
 * launched (100, 75 or 50 % of those that fit; fewer teams share the L1 and L2 among fewer
 * walks). best_wpt, best_occupancy_pct (host int), ms_wpt (host float[4], as for
 * treeray_autotune) and ms_occupancy (host float[3], for 100, 75, 50 %) may be NULL.
 * The choice is kept by the context and remembered for the process, keyed by the tree's
 * shape (leaf count, depth, N_pix, segments, thin or thick tiles, kernel variant, AMR or
 * uniform, device): a later treeray_build of a tree of the same shape, in any context,
 * starts from it without timing. Synchronous.
 */
treeray_status treeray_autotune_launch(treeray_t ctx, int64_t n_sample, int* best_wpt, int* best_occupancy_pct,
                                       float* ms_wpt, float* ms_occupancy, treeray_stream_t stream);
/* The evaluate kernel's current launch choices (host ints, either may be NULL). */
treeray_status treeray_get_launch_config(treeray_t ctx, int* wpt, int* occupancy_pct);
/* Resident teams per SM launched by the evaluate kernel, in % of those that fit (1..100). */
treeray_status treeray_set_occupancy(treeray_t ctx, int occupancy_pct);

/* Set the evaluate kernel's warps per target (2, 3, 4 or 8) by hand; 4 is the default.
 * Trees with thick material run teams of 3 as teams of 4. */
treeray_status treeray_set_warps_per_target(treeray_t ctx, int wpt);

/*
 * Batches: many independent boxes (contexts with built trees, the same npix and nbins,
 * any grids and parameters otherwise) evaluated by one persistent launch whose work
 * counter spans the targets of all boxes, so uneven boxes balance across the GPU.
 * A batch records the boxes' trees and ray orientations when created; rebuilding a box or
 * changing its orientations invalidates it (destroy and create again). Contexts must
 * outlive the batch.
 */
typedef struct treeray_batch* treeray_batch_t;
treeray_status treeray_batch_create(const treeray_t* ctxs, int n_boxes, treeray_batch_t* out);
treeray_status treeray_batch_destroy(treeray_batch_t batch);
/*
 * Evaluate every leaf of every box (Secs. 4.2-4.4, as treeray_evaluate with targets NULL).
 *  J, F       host arrays of n_boxes device pointers: J[k] float[N_k], F[k] double[3 N_k].
 *  use_graph  1: the launch is captured once into a CUDA graph (per set of output
 *             pointers) and replayed; 0: plain launch.
 */
treeray_status treeray_batch_evaluate(treeray_batch_t batch, float* const* J, double* const* F,
                                      int use_graph, treeray_stream_t stream);

/*
 * Learned warm start of the fixed point. The paper has no learned component; a small
 * network predicts log10 T_d per cell from 6 features, and the fixed point still decides
 * the result (treeray_fixed_point from the predicted temperatures).
 *
 * Features (treeray_features), per leaf, 6 floats, row-major X[N][6]:
 *   log10 rho, log10 T_gas, log10(mean over rays of the ray optical depth + 1e-6),
 *   log10(ionising photon flux + 1), log10(smallest ray optical depth + 1e-6),
 *   log10(J + 1e-30) with J the mean intensity of this same evaluation (stars included).
 * treeray_features runs one ray evaluation of the current tree (J, F as treeray_evaluate,
 * plus tau_mean, tau_min: device float[N]) and then fills X (device float[6N]).
 * phi: device float[N] ionising photon flux or NULL (zero).
 */
treeray_status treeray_features(treeray_t ctx, const float* Tgas, const float* phi, float* X, float* J,
                                double* F, float* tau_mean, float* tau_min, treeray_stream_t stream);

/*
 * The network: 6 -> 64 -> 64 -> 1 with SiLU activations; FP32 master weights, BF16 weights
 * and BF16-rounded layer inputs multiplied with FP32 accumulation. Parameters are a flat
 * float[4673]: W1[64][6], b1[64], W2[64][64], b2[64], W3[64], b3[1]. The normalisation
 * norm[14]: feature means [0..5], feature std [6..11], target mean [12], target std [13];
 * the network maps normalised features to the normalised target log10 T_d.
 */
typedef struct treeray_mlp* treeray_mlp_t;
/* Glorot-uniform weights from seed (host generator), zero biases, identity normalisation. */
treeray_status treeray_mlp_create(uint64_t seed, treeray_mlp_t* out);
treeray_status treeray_mlp_destroy(treeray_mlp_t mlp);
/* Host float[4673] parameters and/or float[14] normalisation (either may be NULL); setting
 * parameters resets the optimiser state. get copies them out. Synchronous. */
treeray_status treeray_mlp_set_params(treeray_mlp_t mlp, const float* params, const float* norm);
treeray_status treeray_mlp_get_params(treeray_mlp_t mlp, float* params, float* norm);
/* Normalisation from data: column means and standard deviations of X (device float[6n])
 * and y (device float[n], log10 T_d). */
treeray_status treeray_mlp_fit_normalization(treeray_mlp_t mlp, const float* X, const float* y, int64_t n,
                                             treeray_stream_t stream);
/*
 * Adam training (beta 0.9 / 0.999, eps 1e-8) on the mean-square error of the normalised
 * target: `steps` minibatches of `batch` samples drawn with replacement by a counter-based
 * hash of (seed, step, slot) (splitmix64); loss_history host float[steps] (mean batch loss
 * before each update) or NULL. X device float[6n], y device float[n]. Synchronous when
 * loss_history is given.
 */
treeray_status treeray_mlp_train(treeray_mlp_t mlp, const float* X, const float* y, int64_t n, int batch,
                                 int steps, float lr, uint64_t seed, float* loss_history,
                                 treeray_stream_t stream);
/* Gradient of the mean loss over all n samples (in order) with respect to the 4673
 * parameters, to host float[4673]; host *loss the mean loss. Synchronous. */
treeray_status treeray_mlp_grad(treeray_mlp_t mlp, const float* X, const float* y, int64_t n, float* grad,
                                float* loss, treeray_stream_t stream);
/* Predicted log10 T_d for n feature rows (tensor cores, mma m16n8k16 BF16 -> FP32).
 * X device float[6n], y device float[n]. */
treeray_status treeray_mlp_infer(treeray_mlp_t mlp, const float* X, int64_t n, float* y,
                                 treeray_stream_t stream);
/* Td (device float[N]) = max(2.7 K, 10^prediction) for the leaves' features X (float[6N]). */
treeray_status treeray_warm_start(treeray_t ctx, treeray_mlp_t mlp, const float* X, float* Td,
                                  treeray_stream_t stream);

/* Synchronize the stream and report errors recorded by kernels since the last check
 * (TREERAY_ETIMEOUT for a bounded loop that ran out, such as a walk stack that would have
 * overflowed; TREERAY_EINVAL for a target index out of range or an input field with a
 * negative or non-finite value; TREERAY_ECUDA for CUDA errors). Clears the record. */
treeray_status treeray_check(treeray_t ctx, treeray_stream_t stream);

/* Number of leaves and nodes of the current tree (0 before a build). */
int64_t treeray_leaf_count(treeray_t ctx);
int64_t treeray_node_count(treeray_t ctx);

/*
 * Copy the tree to HOST arrays, nodes breadth first (level-major, Morton order within
 * a level), for structure and moment checks. Any pointer may be NULL.
 *  level int32[nn]; leaf int32[nn] (caller leaf index, -1 for h-nodes);
 *  child0 int32[nn] (first sub-node id, -1 for leaves); centre int64[3nn] (geometric
 *  centre in half-cells of the finest level); vals double[11nn] per node: thin L (+S),
 *  thin A~, thin V, thick sum L_ V, thick A~, thick V, mass, xi, COL xyz (half-cells).
 * Synchronizes the stream.
 */
treeray_status treeray_tree_export(treeray_t ctx, int32_t* level, int32_t* leaf, int32_t* child0,
                                   int64_t* centre, double* vals, treeray_stream_t stream);

/* Copy per-leaf build outputs to HOST double arrays (caller order): kappa, tau_b, J_src,
 * P_src, and int32 thick flags. Any pointer may be NULL. Synchronizes the stream. */
treeray_status treeray_leaf_export(treeray_t ctx, double* kappa, double* tau, double* jsrc,
                                   double* psrc, int32_t* thick, treeray_stream_t stream);

/*
 * Accepted-node lists of the walk (structure check; slow, one warp per target).
 *  targets device int32[n] caller leaf indices; counts device int32[n] receives each
 *  target's number of accepted nodes; ids device int32[n * cap] receives the first
 *  cap node ids of target q at ids[q * cap], in walk order.
 */
treeray_status treeray_accepted(treeray_t ctx, const int32_t* targets, int64_t n, int32_t cap,
                                int32_t* counts, int32_t* ids, treeray_stream_t stream);

/*
 * Walk statistics for the roofline model: totals over the targets of nodes visited
 * (tested against the opening criterion), nodes accepted (own cell included) and
 * angular-kernel entries read. targets device int32[n] or NULL for every leaf;
 * totals device int64[3], accumulated (the caller zeroes it).
 */
treeray_status treeray_walk_stats(treeray_t ctx, const int32_t* targets, int64_t n,
                                  int64_t* totals, treeray_stream_t stream);

/*
 * Morton ordering of the leaves without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc, such
 * as a host simulation code whose own pool allocator owns all device memory and
 * forbids allocations by the libraries it links, or a caller issuing work from a
 * region where allocation is not allowed. It computes the same ordering as the first
 * step of treeray_build (Morton key of each leaf's lower corner at the finest level,
 * prefixed by the leaf's level; stable radix sort) and needs no context.
 *  grid   as for treeray_build, at most 524288 leaves (AMR: at most 1024 blocks);
 *         larger grids return TREERAY_EINVAL.
 *  keys   device uint64[N] output, sorted keys (level << 3 lmax | Morton code).
 *  perm   device int32[N] output, caller leaf index of each sorted position.
 *         The caller sizes both outputs to the leaf count N (n^3, or 512 per AMR
 *         block); the library cannot check their length.
 * An AMR grid's block table is copied from host memory on each call, which a stream
 * capture cannot record: for AMR grids this call returns TREERAY_EINVAL while the
 * stream is being captured (uniform grids need no host copy).
 * All scratch memory (6.2 MiB) is one fixed device array inside the library, held by
 * every GPU that loads the library until the process exits. The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress), so make the
 * first call on each device before any stream capture. Every call shares the array
 * and it keeps the last call's contents; calls whose work overlaps on the GPU (on
 * different streams, or from different threads) race on it, so serialise them.
 */
treeray_status treeray_morton_order_noalloc(const treeray_grid* grid, uint64_t* keys,
                                            int32_t* perm, treeray_stream_t stream);

/*
 * Host-only: angular-kernel hit counts of key K (three ints) for npix rays and s samples
 * per axis, written to counts[npix]. Needs no GPU; used to check the table builder.
 */
treeray_status treeray_alpha_counts_host(int npix, int s, const int64_t* K, int32_t* counts);

/* Host-only: the same counts for the ray set turned by the row-major rotation rot[9]
 * (Sec. 7.6, several orientations): sample direction v counts in the pixel of R^T v. */
treeray_status treeray_alpha_counts_rotated_host(int npix, int s, const int64_t* K, const double* rot,
                                                 int32_t* counts);

/* Number of CUDA kernels this context has launched since it was created
 * (instrumentation for benchmarks; counted on the host at each launch). */
int64_t treeray_kernel_launches(treeray_t ctx);

/*
 * Test hooks for the error paths (no counterpart in the paper; they change no result when
 * left at 0).
 *  treeray_set_walk_stack_limit: cap the evaluation walk's stack at `entries` child groups
 *    (0: the full stack, sized for the tree's depth). A walk that needs more stops for that
 *    target, records a stack overflow in the device error word and returns normally;
 *    treeray_check then reports TREERAY_ETIMEOUT. That target's J and F are not written.
 *  treeray_inject_alloc_failure: the n-th device allocation made by this context from now
 *    on fails as if the device were out of memory (n >= 1; 0 disables); the call that makes
 *    it returns TREERAY_ENOMEM, leaves the context without a tree (TREERAY_ENOTBUILT until
 *    the next successful treeray_build) and destroyable.
 */
treeray_status treeray_set_walk_stack_limit(treeray_t ctx, int entries);
treeray_status treeray_inject_alloc_failure(treeray_t ctx, int n);

/* Message of the last error on this thread (empty string if none). */
const char* treeray_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TREERAY_H */
