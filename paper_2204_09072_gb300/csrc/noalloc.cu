// Morton ordering of the leaves that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host simulation code that hands all device
// memory to its own pool allocator and forbids allocations by libraries it links, or a
// caller that issues its work from a region where allocation is not allowed. This
// file gives them the leaf ordering step of the tree build (the same Morton keys and
// stable LSD radix sort as treeray_build) with every piece of scratch memory in one
// file-scope device array of fixed size, kNoAllocBytes below. Every GPU that loads the
// library holds that array until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device address: the
// device address is looked up once per device with cudaGetSymbolAddress (with that
// device current) on the first call made on that device, and passed to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace tr {
namespace {

constexpr int64_t kNoAllocMaxLeaves = (int64_t)1 << 19;   // 524288 leaves (e.g. 64^3 = 262144)
constexpr int kNaTile = 4096;                              // keys per block and pass
constexpr int kNaThreads = 256;
constexpr int64_t kNaMaxBlocks = kNoAllocMaxLeaves / kNaTile;                 // 128
constexpr int64_t kNaMaxAmrBlocks = kNoAllocMaxLeaves / 512;                  // 1024
// layout: keys [max] u64 | vals [max] i32 | histogram [256 x max blocks] u32 | AMR blocks
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = kOffKeys + 8 * (size_t)kNoAllocMaxLeaves;
constexpr size_t kOffHist = kOffVals + 4 * (size_t)kNoAllocMaxLeaves;
constexpr size_t kOffBlocks = kOffHist + 4 * 256 * (size_t)kNaMaxBlocks;
constexpr size_t kNoAllocBytes = kOffBlocks + 16 * (size_t)kNaMaxAmrBlocks;  // 6.16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[kMaxDevices] = {nullptr};

__device__ inline uint64_t na_morton(uint64_t x, uint64_t y, uint64_t z, int bits) {
    uint64_t k = 0;
    for (int b = 0; b < bits; ++b)
        k |= (((x >> b) & 1ull) << (3 * b)) | (((y >> b) & 1ull) << (3 * b + 1)) |
             (((z >> b) & 1ull) << (3 * b + 2));
    return k;
}

__global__ void na_keys(int n, int lmax, const int4* blocks, int64_t count, uint64_t* keys, int32_t* vals) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= count) return;
    int64_t c[3];
    int l;
    if (n > 0) {
        c[0] = k % n;
        c[1] = (k / n) % n;
        c[2] = k / ((int64_t)n * n);
        l = lmax;
    } else {
        const int4 b = blocks[k >> 9];
        const int q = (int)(k & 511);
        c[0] = 8 * (int64_t)b.x + (q & 7);
        c[1] = 8 * (int64_t)b.y + ((q >> 3) & 7);
        c[2] = 8 * (int64_t)b.z + (q >> 6);
        l = b.w;
    }
    const int sh = lmax - l;
    keys[k] = ((uint64_t)l << (3 * lmax)) |
              na_morton((uint64_t)c[0] << sh, (uint64_t)c[1] << sh, (uint64_t)c[2] << sh, lmax);
    vals[k] = (int32_t)k;
}

// every (digit, block) counter is written, so the histogram needs no clearing
__global__ void na_hist(const uint64_t* keys, int64_t n, int shift, uint32_t* hist, int nb) {
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kNaTile;
    for (int j = threadIdx.x; j < kNaTile; j += blockDim.x) {
        const int64_t i = base + j;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * nb + blockIdx.x] = h[d];
}

__global__ void na_scan(uint32_t* a, int64_t m) {
    __shared__ uint32_t part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (m + 1023) / 1024;
    const int64_t lo = t * chunk, hi = min(m, lo + chunk);
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += a[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - s;
    for (int64_t i = lo; i < hi; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(kNaThreads) na_scatter(const uint64_t* kin, const int32_t* vin,
                                                         uint64_t* kout, int32_t* vout, int64_t n,
                                                         int shift, const uint32_t* hist, int nb) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wc[kNaThreads / 32][257];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int d = t; d < 256; d += blockDim.x) base[d] = hist[(int64_t)d * nb + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int c = 0; c < kNaTile / kNaThreads; ++c) {
        for (int i = t; i < (kNaThreads / 32) * 257; i += blockDim.x) (&wc[0][0])[i] = 0;
        __syncthreads();
        const int64_t i = (int64_t)blockIdx.x * kNaTile + (int64_t)c * kNaThreads + t;
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
            for (int w = 0; w < kNaThreads / 32; ++w) tot += wc[w][dd];
            base[dd] += tot;
        }
        __syncthreads();
    }
}

// Device address of the scratch array on the current device, looked up on the first
// call made on that device.
treeray_status scratch_ptr(unsigned char** out) {
    int dev = 0;
    TR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("morton_order_noalloc: device index out of range");
        return TREERAY_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("morton_order_noalloc: cudaGetSymbolAddress failed: ") +
                      cudaGetErrorString(e));
            return TREERAY_ECUDA;
        }
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_na_ptr[dev];
    return TREERAY_OK;
}

}  // namespace
}  // namespace tr

using namespace tr;

extern "C" treeray_status treeray_morton_order_noalloc(const treeray_grid* g, uint64_t* keys,
                                                       int32_t* perm, treeray_stream_t stream) {
    if (!g || !keys || !perm) {
        set_error("morton_order_noalloc: grid, keys and perm are required");
        return TREERAY_EINVAL;
    }
    int lmax = 0;
    int64_t N = 0;
    int4 hb[kNaMaxAmrBlocks];
    if (g->n < 0) {
        set_error("morton_order_noalloc: n must be a power of two (uniform) or 0 (AMR blocks)");
        return TREERAY_EINVAL;
    }
    if (g->n > 0) {
        if (g->n_blocks != 0) {
            set_error("morton_order_noalloc: give either n (uniform) or n_blocks (AMR), not both");
            return TREERAY_EINVAL;
        }
        while ((1 << lmax) < g->n) ++lmax;
        if ((1 << lmax) != g->n || lmax > 10) {
            set_error("morton_order_noalloc: n must be a power of two <= 1024");
            return TREERAY_EINVAL;
        }
        N = (int64_t)g->n * g->n * g->n;
    } else {
        if (g->n_blocks <= 0 || !g->blocks) {
            set_error("morton_order_noalloc: n_blocks must be positive with a host blocks array");
            return TREERAY_EINVAL;
        }
        if (g->n_blocks > kNaMaxAmrBlocks) {
            set_error("morton_order_noalloc: at most 1024 AMR blocks (524288 leaves)");
            return TREERAY_EINVAL;
        }
        for (int b = 0; b < g->n_blocks; ++b) {
            const int32_t* q = g->blocks + 4 * b;
            if (q[3] < 3 || q[3] > kMaxLevel) {
                set_error("morton_order_noalloc: AMR cell levels must lie in 3..19");
                return TREERAY_EINVAL;
            }
            const int64_t nb = (int64_t)1 << (q[3] - 3);
            for (int a = 0; a < 3; ++a)
                if (q[a] < 0 || q[a] >= nb) {
                    set_error("morton_order_noalloc: AMR block coordinates outside the box");
                    return TREERAY_EINVAL;
                }
            hb[b] = make_int4(q[0], q[1], q[2], q[3]);
            lmax = std::max(lmax, (int)q[3]);
        }
        N = (int64_t)g->n_blocks * 512;
    }
    if (N > kNoAllocMaxLeaves) {
        set_error("morton_order_noalloc: at most 524288 leaves (the fixed scratch size)");
        return TREERAY_EINVAL;
    }
    unsigned char* scratch = nullptr;
    treeray_status rc = scratch_ptr(&scratch);
    if (rc != TREERAY_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t* kalt = reinterpret_cast<uint64_t*>(scratch + kOffKeys);
    int32_t* valt = reinterpret_cast<int32_t*>(scratch + kOffVals);
    uint32_t* hist = reinterpret_cast<uint32_t*>(scratch + kOffHist);
    int4* dblocks = reinterpret_cast<int4*>(scratch + kOffBlocks);
    if (g->n == 0) {
        // a pageable host copy cannot be recorded into a stream capture
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        TR_CUDA(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            set_error("morton_order_noalloc: AMR grids copy their block table from the host and cannot be captured");
            return TREERAY_EINVAL;
        }
        // the host table is staged through pageable memory: the copy has completed
        // (from the host's point of view) when cudaMemcpyAsync returns
        TR_CUDA(cudaMemcpyAsync(dblocks, hb, sizeof(int4) * g->n_blocks, cudaMemcpyHostToDevice, st));
    }
    const int nbk = (int)((N + kNaTile - 1) / kNaTile);
    const int64_t nh = 256 * (int64_t)nbk;
    na_keys<<<(int)((N + 255) / 256), 256, 0, st>>>(g->n, lmax, dblocks, N, keys, perm);
    uint64_t* ka = keys;
    int32_t* va = perm;
    uint64_t* kb = kalt;
    int32_t* vb = valt;
    int passes = 0;
    for (int shift = 0; shift < 3 * lmax + 5; shift += 8, ++passes) {
        na_hist<<<nbk, kNaThreads, 0, st>>>(ka, N, shift, hist, nbk);
        na_scan<<<1, 1024, 0, st>>>(hist, nh);
        na_scatter<<<nbk, kNaThreads, 0, st>>>(ka, va, kb, vb, N, shift, hist, nbk);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {
        TR_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * N, cudaMemcpyDeviceToDevice, st));
        TR_CUDA(cudaMemcpyAsync(perm, va, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
    }
    TR_CUDA(cudaGetLastError());
    return TREERAY_OK;
}
