// Graph orientation for k-clique counting (Sec. 6.4.2): every undirected edge
// is oriented from the lower to the higher vertex of the order (degree, id),
// giving a DAG in which each k-clique appears exactly once; out-lists are
// sorted by vertex id.  Runs as plain data-parallel kernels before the
// task-parallel count (the paper times both together).
#include <cuda_runtime.h>

#include "gtap.h"
#include "gtap_internal.h"

namespace gtap {
namespace {

__global__ void k_degrees(const int32_t* edges, int64_t m, int32_t* deg) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(&deg[edges[2 * e]], 1);
        atomicAdd(&deg[edges[2 * e + 1]], 1);
    }
}

__device__ __forceinline__ bool before(const int32_t* deg, int32_t a, int32_t b) {
    const int32_t da = deg[a], db = deg[b];
    return da != db ? da < db : a < b;
}

__global__ void k_outdeg(const int32_t* edges, int64_t m, const int32_t* deg, int32_t* outdeg) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        atomicAdd(&outdeg[before(deg, a, b) ? a : b], 1);
    }
}

// Exclusive scan of n int32 counts into n+1 int64 offsets: per-block scans, a
// scan of the block sums in one block, then the block offsets are added.
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* sh, long long* total) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        long long s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const long long warp_prefix = (w > 0) ? sh[w - 1] : 0;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

__global__ void k_scan_tiles(const int32_t* cnt, int64_t n, int64_t* off, long long* tile_sums) {
    __shared__ long long sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long v[kScanItems], s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) { v[i] = (base + i < n) ? cnt[base + i] : 0; s += v[i]; }
    long long total;
    long long ex = block_exclusive_scan(s, sh, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) { if (base + i < n) off[base + i] = ex; ex += v[i]; }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(long long* tile_sums, int ntiles, int64_t* off, int64_t n) {
    __shared__ long long sh[32];
    long long carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += blockDim.x) {
        const int i = b0 + threadIdx.x;
        const long long v = (i < ntiles) ? tile_sums[i] : 0;
        long long total;
        const long long ex = block_exclusive_scan(v, sh, &total);
        if (i < ntiles) tile_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) off[n] = carry;
}

__global__ void k_scan_add(int64_t* off, int64_t n, const long long* tile_sums) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        off[i] += tile_sums[i / kScanTile];
}

__global__ void k_scatter(const int32_t* edges, int64_t m, const int32_t* deg, const int64_t* off, int32_t* cursor,
                          int32_t* adj) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = edges[2 * e], b = edges[2 * e + 1];
        const bool ab = before(deg, a, b);
        const int32_t x = ab ? a : b, y = ab ? b : a;
        const int32_t pos = atomicAdd(&cursor[x], 1);
        adj[off[x] + pos] = y;
    }
}

// Sort short out-lists (<= 32) with one warp each (bitonic over lanes); longer
// lists are collected for the block sorter.
__global__ void k_sort_small(const int64_t* off, int64_t n, int32_t* adj, int32_t* big, int32_t* nbig) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < n; x += nwarps) {
        const int64_t b = off[x];
        const int len = (int)(off[x + 1] - b);
        if (len <= 1) continue;
        if (len > 32) {
            if (lane == 0) big[atomicAdd(nbig, 1)] = (int32_t)x;
            continue;
        }
        int v = (lane < len) ? adj[b + lane] : 0x7FFFFFFF;
        for (int k = 2; k <= 32; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int o = __shfl_xor_sync(0xffffffffu, v, j);
                const bool up = (lane & k) == 0;
                const bool lower = (lane & j) == 0;
                v = (lower == up) ? min(v, o) : max(v, o);
            }
        }
        if (lane < len) adj[b + lane] = v;
    }
}

// One block sorts each long out-list in shared memory (bitonic, padded to a power of two).
constexpr int kBigSort = 8192;
__global__ void k_sort_big(const int64_t* off, int32_t* adj, const int32_t* big, const int32_t* nbig, int* status) {
    __shared__ int s[kBigSort];
    const int cnt = *nbig;
    for (int bi = blockIdx.x; bi < cnt; bi += gridDim.x) {
        const int32_t x = big[bi];
        const int64_t b = off[x];
        const int len = (int)(off[x + 1] - b);
        if (len > kBigSort) {
            if (threadIdx.x == 0) atomicMax(status, len);
            continue;
        }
        int np = 1;
        while (np < len) np <<= 1;
        for (int i = threadIdx.x; i < np; i += blockDim.x) s[i] = (i < len) ? adj[b + i] : 0x7FFFFFFF;
        __syncthreads();
        for (int k = 2; k <= np; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int p = threadIdx.x; p < (np >> 1); p += blockDim.x) {
                    const int i = 2 * j * (p / j) + (p % j);
                    const int q = i + j;
                    const int a = s[i], c = s[q];
                    const bool up = (i & k) == 0;
                    if ((a > c) == up) { s[i] = c; s[q] = a; }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < len; i += blockDim.x) adj[b + i] = s[i];
        __syncthreads();
    }
}

__global__ void k_sources(const int64_t* off, int64_t n, int32_t* src) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < n; x += nwarps)
        for (int64_t e = off[x] + lane; e < off[x + 1]; e += 32) src[e] = (int32_t)x;
}

}  // namespace
}  // namespace gtap

using namespace gtap;

extern "C" gtap_status gtap_kclique_orient(const int32_t* edges, int64_t m, int64_t n, int64_t* off, int32_t* adj,
                                           int32_t* src, int32_t* work, void* stream) {
    if (m < 0 || n < 1 || n >= (1ll << 31) || m >= (1ll << 31)) return GTAP_ERR_INVALID_ARG;
    if (!off || !work || (m > 0 && (!edges || !adj || !src))) return GTAP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // work layout: deg[n] | outdeg/cursor[n] | big list[n] | counters (2 ints) | tile sums (int64, aligned)
    int32_t* deg = work;
    int32_t* cnt = work + n;
    int32_t* big = work + 2 * n;
    int32_t* nbig = work + 3 * n;
    int32_t* status = nbig + 1;
    long long* tile_sums = reinterpret_cast<long long*>(work + 3 * n + 2 + ((3 * n + 2) & 1));
    const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
    const int g = 1024;
    if (cudaMemsetAsync(work, 0, (size_t)(3 * n + 2) * sizeof(int32_t), st) != cudaSuccess) return GTAP_ERR_CUDA;
    if (m > 0) {
        k_degrees<<<g, 256, 0, st>>>(edges, m, deg);
        k_outdeg<<<g, 256, 0, st>>>(edges, m, deg, cnt);
    }
    k_scan_tiles<<<ntiles, kScanBlock, 0, st>>>(cnt, n, off, tile_sums);
    k_scan_sums<<<1, kScanBlock, 0, st>>>(tile_sums, ntiles, off, n);
    k_scan_add<<<g, 256, 0, st>>>(off, n, tile_sums);
    if (cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int32_t), st) != cudaSuccess) return GTAP_ERR_CUDA;
    if (m > 0) {
        k_scatter<<<g, 256, 0, st>>>(edges, m, deg, off, cnt, adj);
        k_sort_small<<<g, 256, 0, st>>>(off, n, adj, big, nbig);
        k_sort_big<<<304, 512, 0, st>>>(off, adj, big, nbig, status);
        k_sources<<<g, 256, 0, st>>>(off, n, src);
    }
    if (cudaGetLastError() != cudaSuccess) return GTAP_ERR_CUDA;
    int bad = 0;
    if (cudaMemcpyAsync(&bad, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GTAP_ERR_CUDA;
    return bad ? GTAP_ERR_INVALID_ARG : GTAP_OK;
}
