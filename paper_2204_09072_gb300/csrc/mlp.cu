// Learned warm start of the dust-temperature fixed point: a 6 -> 64 -> 64 -> 1 SiLU
// multilayer perceptron predicting log10 T_d from per-cell features (log density, log gas
// temperature, log mean and smallest ray optical depth, log ionising flux, log J of the
// feature pass at the initial dust temperatures). The paper has no learned component; this network only sets
// the starting point of the iteration, which still converges to the same fixed point.
//
// Numerics: FP32 master weights; BF16 copies of the weights and BF16-rounded layer
// inputs (normalised features and activations) are multiplied with FP32 accumulation.
//   inference:  tensor cores, mma.sync m16n8k16 (BF16 in, FP32 accumulate); each warp
//               runs 16 cells through all three layers; the accumulator fragments of one
//               layer are, after SiLU and BF16 packing, the A fragments of the next.
//   training:   one thread per sample for the forward and per-sample backward passes,
//               weight gradients reduced over the batch per output row (deterministic),
//               Adam on the FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <random>
#include <vector>

#include "internal.h"

namespace tr {
namespace {

constexpr int kIn = 6, kHid = 64;
constexpr int oW1 = 0, oB1 = oW1 + kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kHid, kParams = oB3 + 1;  // 4673

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// normalisation: norm[0..5] feature means, [6..11] feature std, [12] target mean, [13] target std
__device__ __forceinline__ float xnorm(const float* norm, float x, int i) { return (x - norm[i]) / norm[6 + i]; }

__device__ __forceinline__ void mma_bf16(float& c0, float& c1, float& c2, float& c3, uint32_t a0, uint32_t a1,
                                         uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------- inference
// Shared-memory weight layout (BF16): W1 as [64][16] (inputs padded with zeros), W2 [64][64],
// W3 as [8][64] (rows 1..7 zero); biases FP32.
struct __align__(16) TcSmem {
    __nv_bfloat16 w1[kHid][16];
    __nv_bfloat16 w2[kHid][kHid];
    __nv_bfloat16 w3[8][kHid];
    float b1[kHid], b2[kHid], b3;
    float norm[14];
};

__global__ void __launch_bounds__(256) k_mlp_infer_tc(const __nv_bfloat16* __restrict__ wb,
                                                      const float* __restrict__ params,
                                                      const float* __restrict__ norm, const float* __restrict__ X,
                                                      int64_t n, float* __restrict__ y) {
    __shared__ TcSmem sm;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < kHid * 16; i += blockDim.x) {
        const int r = i / 16, c = i % 16;
        sm.w1[r][c] = c < kIn ? wb[oW1 + r * kIn + c] : __float2bfloat16_rn(0.0f);
    }
    for (int i = tid; i < kHid * kHid; i += blockDim.x) sm.w2[i / kHid][i % kHid] = wb[oW2 + i];
    for (int i = tid; i < 8 * kHid; i += blockDim.x)
        sm.w3[i / kHid][i % kHid] = i < kHid ? wb[oW3 + i] : __float2bfloat16_rn(0.0f);
    for (int i = tid; i < kHid; i += blockDim.x) {
        sm.b1[i] = params[oB1 + i];
        sm.b2[i] = params[oB2 + i];
    }
    if (tid == 0) sm.b3 = params[oB3];
    if (tid < 14) sm.norm[tid] = norm[tid];
    __syncthreads();
    const int g = lane >> 2, t4 = lane & 3;
    const int64_t tiles = (n + 15) / 16;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + tid) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tile = wid; tile < tiles; tile += nw) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        // layer-1 A fragment: columns 2 t4, 2 t4 + 1 of the 6 normalised features
        float x00 = 0.0f, x01 = 0.0f, x10 = 0.0f, x11 = 0.0f;
        const int c0 = 2 * t4;
        if (c0 < kIn) {
            if (r0 < n) {
                x00 = xnorm(sm.norm, X[r0 * kIn + c0], c0);
                x01 = xnorm(sm.norm, X[r0 * kIn + c0 + 1], c0 + 1);
            }
            if (r1 < n) {
                x10 = xnorm(sm.norm, X[r1 * kIn + c0], c0);
                x11 = xnorm(sm.norm, X[r1 * kIn + c0 + 1], c0 + 1);
            }
        }
        const uint32_t a0 = pack2(x00, x01), a1 = pack2(x10, x11), a2 = 0u, a3 = 0u;
        float h[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = 8 * j + 2 * t4;
            float d0 = sm.b1[col], d1 = sm.b1[col + 1], d2 = d0, d3 = d1;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&sm.w1[8 * j + g][2 * t4]);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&sm.w1[8 * j + g][2 * t4 + 8]);
            mma_bf16(d0, d1, d2, d3, a0, a1, a2, a3, b0, b1);
            h[j][0] = silu(d0);
            h[j][1] = silu(d1);
            h[j][2] = silu(d2);
            h[j][3] = silu(d3);
        }
        // layer 2: K = 64 in four steps of 16; A fragments straight from the layer-1 results
        float o[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = 8 * j + 2 * t4;
            o[j][0] = sm.b2[col];
            o[j][1] = sm.b2[col + 1];
            o[j][2] = o[j][0];
            o[j][3] = o[j][1];
        }
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const uint32_t p0 = pack2(h[2 * ks][0], h[2 * ks][1]);
            const uint32_t p1 = pack2(h[2 * ks][2], h[2 * ks][3]);
            const uint32_t p2 = pack2(h[2 * ks + 1][0], h[2 * ks + 1][1]);
            const uint32_t p3 = pack2(h[2 * ks + 1][2], h[2 * ks + 1][3]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&sm.w2[8 * j + g][16 * ks + 2 * t4]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&sm.w2[8 * j + g][16 * ks + 2 * t4 + 8]);
                mma_bf16(o[j][0], o[j][1], o[j][2], o[j][3], p0, p1, p2, p3, b0, b1);
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) o[j][q] = silu(o[j][q]);
        // layer 3: one output column (N padded to 8)
        float y0 = t4 == 0 ? sm.b3 : 0.0f, y1 = 0.0f, y2 = y0, y3 = 0.0f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const uint32_t p0 = pack2(o[2 * ks][0], o[2 * ks][1]);
            const uint32_t p1 = pack2(o[2 * ks][2], o[2 * ks][3]);
            const uint32_t p2 = pack2(o[2 * ks + 1][0], o[2 * ks + 1][1]);
            const uint32_t p3 = pack2(o[2 * ks + 1][2], o[2 * ks + 1][3]);
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&sm.w3[g][16 * ks + 2 * t4]);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&sm.w3[g][16 * ks + 2 * t4 + 8]);
            mma_bf16(y0, y1, y2, y3, p0, p1, p2, p3, b0, b1);
        }
        if (t4 == 0) {  // column 0 lives in the first thread of each group
            if (r0 < n) y[r0] = y0 * sm.norm[13] + sm.norm[12];
            if (r1 < n) y[r1] = y2 * sm.norm[13] + sm.norm[12];
        }
    }
}

// ----------------------------------------------------------------- training
// Per-sample activations of a training batch, SoA: a0[6] z1[64] a1[64] z2[64] a2[64], dy
constexpr int kAct = kIn + 4 * kHid;

struct FwdSmem {
    float w1[kHid * kIn], w2[kHid * kHid], w3[kHid], b1[kHid], b2[kHid], b3;
    float norm[14];
};

__device__ void load_fwd_smem(FwdSmem& sm, const __nv_bfloat16* wb, const float* params, const float* norm) {
    for (int i = threadIdx.x; i < kHid * kIn; i += blockDim.x) sm.w1[i] = __bfloat162float(wb[oW1 + i]);
    for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x) sm.w2[i] = __bfloat162float(wb[oW2 + i]);
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        sm.w3[i] = __bfloat162float(wb[oW3 + i]);
        sm.b1[i] = params[oB1 + i];
        sm.b2[i] = params[oB2 + i];
    }
    if (threadIdx.x == 0) sm.b3 = params[oB3];
    if (threadIdx.x < 14) sm.norm[threadIdx.x] = norm[threadIdx.x];
    __syncthreads();
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// forward of one batch (one sample per thread); sample ids from a counter-based hash
// (seed, step, slot) when ids == nullptr, else ids[slot]; writes activations and
// dy = (y - t) / B for the mean-square loss (1 / 2B) sum (y - t)^2 on normalised targets
__global__ void __launch_bounds__(128) k_mlp_fwd_train(const __nv_bfloat16* __restrict__ wb,
                                                       const float* __restrict__ params,
                                                       const float* __restrict__ norm, const float* __restrict__ X,
                                                       const float* __restrict__ Y, int64_t n, int B,
                                                       uint64_t seed, int64_t step, float* __restrict__ act,
                                                       float* __restrict__ loss) {
    __shared__ FwdSmem sm;
    load_fwd_smem(sm, wb, params, norm);
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int64_t id = (B == n && seed == 0) ? b
                                             : (int64_t)(splitmix64(seed ^ splitmix64((uint64_t)step * 0x100000001ull + b)) %
                                                         (uint64_t)n);
    float* a = act + (int64_t)b * (kAct + 1);
    float a0[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
        a0[i] = bf16r(xnorm(sm.norm, X[id * kIn + i], i));
        a[i] = a0[i];
    }
    float a1[kHid];
#pragma unroll 4
    for (int j = 0; j < kHid; ++j) {
        float z = sm.b1[j];
        for (int i = 0; i < kIn; ++i) z += sm.w1[j * kIn + i] * a0[i];
        a[kIn + j] = z;
        a1[j] = bf16r(silu(z));
        a[kIn + kHid + j] = a1[j];
    }
    float yv = sm.b3;
    for (int j = 0; j < kHid; ++j) {
        float z = sm.b2[j];
#pragma unroll 8
        for (int i = 0; i < kHid; ++i) z += sm.w2[j * kHid + i] * a1[i];
        a[kIn + 2 * kHid + j] = z;
        const float a2 = bf16r(silu(z));
        a[kIn + 3 * kHid + j] = a2;
        yv += sm.w3[j] * a2;
    }
    const float t = (Y[id] - sm.norm[12]) / sm.norm[13];
    const float dy = (yv - t) / (float)B;
    a[kAct] = dy;
    loss[b] = 0.5f * (yv - t) * (yv - t);
}

// per-sample backward: dz2 = dy w3 silu'(z2), dz1 = (W2^T dz2) silu'(z1); overwrites z1, z2 with dz1, dz2
__global__ void __launch_bounds__(128) k_mlp_bwd_sample(const __nv_bfloat16* __restrict__ wb, int B,
                                                        float* __restrict__ act) {
    __shared__ float w2[kHid * kHid], w3[kHid];
    for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x) w2[i] = __bfloat162float(wb[oW2 + i]);
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) w3[i] = __bfloat162float(wb[oW3 + i]);
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float* a = act + (int64_t)b * (kAct + 1);
    const float dy = a[kAct];
    float dz2[kHid];
#pragma unroll 8
    for (int j = 0; j < kHid; ++j) {
        dz2[j] = dy * w3[j] * dsilu(a[kIn + 2 * kHid + j]);
        a[kIn + 2 * kHid + j] = dz2[j];
    }
    for (int i = 0; i < kHid; ++i) {
        float s = 0.0f;
#pragma unroll 8
        for (int j = 0; j < kHid; ++j) s += w2[j * kHid + i] * dz2[j];
        a[kIn + i] = s * dsilu(a[kIn + i]);
    }
}

// weight gradients, one block per output row: rows 0..63 of W1/b1 (from dz1, a0),
// 64..127 of W2/b2 (from dz2, a1), 128 the W3/b3 row (from dy, a2); sums over the batch
// in a fixed order (deterministic)
__global__ void __launch_bounds__(256) k_mlp_wgrad(const float* __restrict__ act, int B, float* __restrict__ grad) {
    const int row = blockIdx.x;
    int in_off, nin, dz_off, w_off, b_off;
    if (row < kHid) {
        in_off = 0; nin = kIn; dz_off = kIn + row; w_off = oW1 + row * kIn; b_off = oB1 + row;
    } else if (row < 2 * kHid) {
        const int r = row - kHid;
        in_off = kIn + kHid; nin = kHid; dz_off = kIn + 2 * kHid + r; w_off = oW2 + r * kHid; b_off = oB2 + r;
    } else {
        in_off = kIn + 3 * kHid; nin = kHid; dz_off = kAct; w_off = oW3; b_off = oB3;
    }
    __shared__ float part[4][kHid + 1];
    const int t = threadIdx.x, col = t % kHid, chunk = t / kHid;  // 4 chunks of the batch
    float s = 0.0f, sb = 0.0f;
    for (int b = chunk; b < B; b += 4) {
        const float* a = act + (int64_t)b * (kAct + 1);
        const float dz = a[dz_off];
        if (col < nin) s += dz * a[in_off + col];
        if (col == 0) sb += dz;
    }
    part[chunk][col] = s;
    if (col == 0) part[chunk][kHid] = sb;
    __syncthreads();
    if (t < nin) grad[w_off + t] = part[0][t] + part[1][t] + part[2][t] + part[3][t];
    if (t == 0) grad[b_off] = part[0][kHid] + part[1][kHid] + part[2][kHid] + part[3][kHid];
}

__global__ void k_adam(float* p, float* m, float* v, const float* g, __nv_bfloat16* wb, int np, float lr,
                       float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    wb[i] = __float2bfloat16_rn(p[i]);
}

// mean of the per-sample losses of a batch (one block)
__global__ void k_mean_loss(const float* loss, int B, float* out) {
    __shared__ float sh[256];
    float a = 0.0f;
    for (int i = threadIdx.x; i < B; i += blockDim.x) a += loss[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / (float)B;
}

__global__ void k_to_bf16(const float* p, __nv_bfloat16* wb, int np) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) wb[i] = __float2bfloat16_rn(p[i]);
}

// column means and standard deviations (FP64 sums) of X [n x 6] and y; one block per column
__global__ void k_colstats(const float* X, const float* y, int64_t n, float* norm) {
    const int c = blockIdx.x;  // 0..5 features, 6 target
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        const double v = c < kIn ? (double)X[k * kIn + c] : (double)y[k];
        a += v;
        b += v * v;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            s1[threadIdx.x] += s1[threadIdx.x + off];
            s2[threadIdx.x] += s2[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = s1[0] / (double)n;
        const double sd = sqrt(fmax(s2[0] / (double)n - mean * mean, 1e-12));
        if (c < kIn) {
            norm[c] = (float)mean;
            norm[6 + c] = (float)sd;
        } else {
            norm[12] = (float)mean;
            norm[13] = (float)sd;
        }
    }
}

__global__ void k_pow10_floor(const float* y, float* Td, int64_t n) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) Td[k] = fmaxf(exp10f(y[k]), (float)kDustFloorK);
}

}  // namespace
}  // namespace tr

struct treeray_mlp {
    float* p = nullptr;  // FP32 master parameters [4673]
    float* m = nullptr;  // Adam moments
    float* v = nullptr;
    float* g = nullptr;  // gradient
    __nv_bfloat16* wb = nullptr;
    float* norm = nullptr;  // [14]
    float* act = nullptr;   // training batch activations
    float* loss = nullptr;  // per-sample loss of the last batch
    int cap_batch = 0;
    int64_t step = 0;
};

using namespace tr;

namespace {
treeray_status grow_batch(treeray_mlp* m, int B) {
    if (m->cap_batch >= B) return TREERAY_OK;
    if (m->act) cudaFree(m->act);
    if (m->loss) cudaFree(m->loss);
    m->act = nullptr;
    m->loss = nullptr;
    m->cap_batch = 0;
    TR_CUDA(cudaMalloc(&m->act, sizeof(float) * (kAct + 1) * (size_t)B));
    TR_CUDA(cudaMalloc(&m->loss, sizeof(float) * (size_t)B));
    m->cap_batch = B;
    return TREERAY_OK;
}

// one training step (or, with lr = 0 and no update, a gradient evaluation)
treeray_status train_step(treeray_mlp* m, const float* X, const float* Y, int64_t n, int B, uint64_t seed,
                          int64_t step, cudaStream_t s) {
    const int nb = (B + 127) / 128;
    k_mlp_fwd_train<<<nb, 128, 0, s>>>(m->wb, m->p, m->norm, X, Y, n, B, seed, step, m->act, m->loss);
    k_mlp_bwd_sample<<<nb, 128, 0, s>>>(m->wb, B, m->act);
    k_mlp_wgrad<<<2 * kHid + 1, 256, 0, s>>>(m->act, B, m->g);
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}
}  // namespace

extern "C" {

treeray_status treeray_mlp_create(uint64_t seed, treeray_mlp_t* out) {
    if (!out) {
        set_error("mlp_create: out required");
        return TREERAY_EINVAL;
    }
    *out = nullptr;
    treeray_mlp* m = new (std::nothrow) treeray_mlp();
    if (!m) {
        set_error("out of host memory");
        return TREERAY_ENOMEM;
    }
    auto fail = [&](treeray_status rc) {
        treeray_mlp_destroy(m);
        return rc;
    };
    if (cudaMalloc(&m->p, sizeof(float) * kParams) != cudaSuccess ||
        cudaMalloc(&m->m, sizeof(float) * kParams) != cudaSuccess ||
        cudaMalloc(&m->v, sizeof(float) * kParams) != cudaSuccess ||
        cudaMalloc(&m->g, sizeof(float) * kParams) != cudaSuccess ||
        cudaMalloc(&m->wb, sizeof(__nv_bfloat16) * kParams) != cudaSuccess ||
        cudaMalloc(&m->norm, sizeof(float) * 14) != cudaSuccess) {
        set_error("mlp_create: device allocation failed");
        return fail(TREERAY_ENOMEM);
    }
    // Glorot-uniform weights, zero biases, identity normalisation
    std::vector<float> h(kParams, 0.0f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int fan_out, int fan_in) {
        const float lim = std::sqrt(6.0f / (float)(fan_in + fan_out));
        std::uniform_real_distribution<float> u(-lim, lim);
        for (int i = 0; i < fan_out * fan_in; ++i) h[off + i] = u(rng);
    };
    fill(oW1, kHid, kIn);
    fill(oW2, kHid, kHid);
    fill(oW3, 1, kHid);
    std::vector<float> nrm(14, 0.0f);
    for (int i = 0; i < 6; ++i) nrm[6 + i] = 1.0f;
    nrm[13] = 1.0f;
    if (cudaMemcpy(m->p, h.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->m, 0, sizeof(float) * kParams) != cudaSuccess ||
        cudaMemset(m->v, 0, sizeof(float) * kParams) != cudaSuccess ||
        cudaMemcpy(m->norm, nrm.data(), sizeof(float) * 14, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("mlp_create: upload failed");
        return fail(TREERAY_ECUDA);
    }
    k_to_bf16<<<(kParams + 255) / 256, 256>>>(m->p, m->wb, kParams);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        set_error("mlp_create: initialisation failed");
        return fail(TREERAY_ECUDA);
    }
    *out = m;
    return TREERAY_OK;
}

treeray_status treeray_mlp_destroy(treeray_mlp_t m) {
    if (!m) return TREERAY_OK;
    void* ptrs[] = {m->p, m->m, m->v, m->g, m->wb, m->norm, m->act, m->loss};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete m;
    return TREERAY_OK;
}

treeray_status treeray_mlp_set_params(treeray_mlp_t m, const float* params, const float* norm) {
    if (!m) {
        set_error("mlp_set_params: null network");
        return TREERAY_EINVAL;
    }
    if (params) {
        TR_CUDA(cudaMemcpy(m->p, params, sizeof(float) * kParams, cudaMemcpyHostToDevice));
        k_to_bf16<<<(kParams + 255) / 256, 256>>>(m->p, m->wb, kParams);
        TR_CUDA(cudaMemset(m->m, 0, sizeof(float) * kParams));
        TR_CUDA(cudaMemset(m->v, 0, sizeof(float) * kParams));
        m->step = 0;
    }
    if (norm) TR_CUDA(cudaMemcpy(m->norm, norm, sizeof(float) * 14, cudaMemcpyHostToDevice));
    TR_CUDA(cudaDeviceSynchronize());
    return TREERAY_OK;
}

treeray_status treeray_mlp_get_params(treeray_mlp_t m, float* params, float* norm) {
    if (!m) {
        set_error("mlp_get_params: null network");
        return TREERAY_EINVAL;
    }
    TR_CUDA(cudaDeviceSynchronize());
    if (params) TR_CUDA(cudaMemcpy(params, m->p, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    if (norm) TR_CUDA(cudaMemcpy(norm, m->norm, sizeof(float) * 14, cudaMemcpyDeviceToHost));
    return TREERAY_OK;
}

treeray_status treeray_mlp_fit_normalization(treeray_mlp_t m, const float* X, const float* y, int64_t n,
                                             treeray_stream_t stream) {
    if (!m || !X || !y || n < 2) {
        set_error("mlp_fit_normalization: network, X, y and n >= 2 required");
        return TREERAY_EINVAL;
    }
    k_colstats<<<kIn + 1, 256, 0, (cudaStream_t)stream>>>(X, y, n, m->norm);
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}

treeray_status treeray_mlp_grad(treeray_mlp_t m, const float* X, const float* y, int64_t n, float* grad,
                                float* loss, treeray_stream_t stream) {
    if (!m || !X || !y || n < 1 || n > (1 << 24)) {
        set_error("mlp_grad: network, X, y and 1 <= n <= 2^24 required");
        return TREERAY_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    treeray_status rc = grow_batch(m, (int)n);
    if (rc != TREERAY_OK) return rc;
    if ((rc = train_step(m, X, y, n, (int)n, 0, 0, s)) != TREERAY_OK) return rc;
    TR_CUDA(cudaStreamSynchronize(s));
    if (grad) TR_CUDA(cudaMemcpy(grad, m->g, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    if (loss) {
        std::vector<float> l(n);
        TR_CUDA(cudaMemcpy(l.data(), m->loss, sizeof(float) * n, cudaMemcpyDeviceToHost));
        double sum = 0.0;
        for (float v : l) sum += v;
        *loss = (float)(sum / (double)n);
    }
    return TREERAY_OK;
}

treeray_status treeray_mlp_train(treeray_mlp_t m, const float* X, const float* y, int64_t n, int batch,
                                 int steps, float lr, uint64_t seed, float* loss_history,
                                 treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_mlp_train");
    if (!m || !X || !y || n < 1 || batch < 1 || batch > (1 << 20) || steps < 0 || !(lr >= 0.0f) || seed == 0) {
        set_error("mlp_train: network, X, y, n >= 1, 1 <= batch <= 2^20, steps >= 0, lr >= 0, seed != 0");
        return TREERAY_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    treeray_status rc = grow_batch(m, batch);
    if (rc != TREERAY_OK) return rc;
    float* hist = nullptr;
    if (loss_history) TR_CUDA(cudaMalloc(&hist, sizeof(float) * std::max(steps, 1)));
    for (int k = 0; k < steps; ++k) {
        ++m->step;
        if ((rc = train_step(m, X, y, n, batch, seed, m->step, s)) != TREERAY_OK) break;
        const float c1 = 1.0f - std::pow(0.9f, (float)m->step), c2 = 1.0f - std::pow(0.999f, (float)m->step);
        k_adam<<<(kParams + 255) / 256, 256, 0, s>>>(m->p, m->m, m->v, m->g, m->wb, kParams, lr, c1, c2);
        if (hist) k_mean_loss<<<1, 256, 0, s>>>(m->loss, batch, hist + k);  // loss before the update
    }
    if (rc == TREERAY_OK && hist) {
        cudaError_t ce = cudaMemcpyAsync(loss_history, hist, sizeof(float) * steps, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        cudaFree(hist);
        TR_CUDA(ce);
    } else if (hist) {
        cudaFree(hist);
    }
    TR_CUDA(cudaGetLastError());
    return rc;
}

treeray_status treeray_mlp_infer(treeray_mlp_t m, const float* X, int64_t n, float* y, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_mlp_infer");
    if (!m || !X || !y || n < 0) {
        set_error("mlp_infer: network, X and y required");
        return TREERAY_EINVAL;
    }
    if (n == 0) return TREERAY_OK;
    int sms = 0, dev = 0;
    TR_CUDA(cudaGetDevice(&dev));
    TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t tiles = (n + 15) / 16;
    const int64_t blocks = std::min<int64_t>((tiles + 7) / 8, (int64_t)sms * 8);
    k_mlp_infer_tc<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(m->wb, m->p, m->norm, X, n, y);
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}

treeray_status treeray_features(treeray_t c, const float* Tgas, const float* phi, float* X, float* J, double* F,
                                float* tau_mean, float* tau_min, treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_features");
    if (!c || !c->built) {
        set_error("features: no tree");
        return c ? TREERAY_ENOTBUILT : TREERAY_EINVAL;
    }
    if (!Tgas || !X || !J || !F || !tau_mean || !tau_min) {
        set_error("features: Tgas, X, J, F, tau_mean and tau_min required");
        return TREERAY_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    treeray_status rc = launch_evaluate_tau(c, J, F, tau_mean, tau_min, s);
    if (rc != TREERAY_OK) return rc;
    return launch_features(c, Tgas, phi, tau_mean, tau_min, J, X, s);
}

treeray_status treeray_warm_start(treeray_t c, treeray_mlp_t m, const float* X, float* Td,
                                  treeray_stream_t stream) {
    NvtxRange nvtx_("treeray_warm_start");
    if (!c || !m || !X || !Td || !c->built) {
        set_error("warm_start: built context, network, features and Td required");
        return TREERAY_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    treeray_status rc = treeray_mlp_infer(m, X, c->nleaves, Td, stream);  // log10 T_d into Td
    if (rc != TREERAY_OK) return rc;
    k_pow10_floor<<<(int)((c->nleaves + 255) / 256), 256, 0, s>>>(Td, Td, c->nleaves);
    c->launches += 2;
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}

}  // extern "C"
