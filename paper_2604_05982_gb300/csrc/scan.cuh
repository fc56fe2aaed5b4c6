// Exclusive prefix sum of int32 counts for the data-parallel FMM kernels:
// per-tile block scans, one block scanning the tile sums, then the tile
// offsets are added.  The length may live on the device (n_dev), so a scan
// can be enqueued before the size it covers is known on the host; n_max
// bounds it and sizes the grid.
#pragma once
#include <cuda_runtime.h>

namespace gtap {
namespace scan {
namespace {   // internal linkage: every translation unit that scans gets its own copy

constexpr int kBlock = 1024;
constexpr int kItems = 4;
constexpr int kTile = kBlock * kItems;

__device__ __forceinline__ long long length(const int* n_dev, long long n_host) {
    return n_dev ? (long long)*n_dev : n_host;
}

// Block-wide exclusive scan of one value per thread; *total receives the sum.
__device__ __forceinline__ int block_excl(int v, int* sh, int* total) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = (int)(blockDim.x >> 5);
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = (lane < nw) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const int prefix = (w > 0) ? sh[w - 1] : 0;
    *total = sh[nw - 1];
    __syncthreads();
    return prefix + x - v;
}

__global__ void __launch_bounds__(kBlock) k_tiles(const int* in, const int* n_dev, long long n_host, int* out,
                                                  int* tile_sums) {
    __shared__ int sh[32];
    const long long n = length(n_dev, n_host);
    const long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kItems;
    if ((long long)blockIdx.x * kTile >= n) {
        if (threadIdx.x == 0) tile_sums[blockIdx.x] = 0;
        return;
    }
    int v[kItems], s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) { v[i] = (base + i < n) ? in[base + i] : 0; s += v[i]; }
    int total;
    int ex = block_excl(s, sh, &total);
#pragma unroll
    for (int i = 0; i < kItems; ++i) { if (base + i < n) out[base + i] = ex; ex += v[i]; }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kBlock) k_sums(int* tile_sums, int ntiles, int* total_out) {
    __shared__ int sh[32];
    int carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += kBlock) {
        const int i = b0 + (int)threadIdx.x;
        const int v = (i < ntiles) ? tile_sums[i] : 0;
        int total;
        const int ex = block_excl(v, sh, &total);
        if (i < ntiles) tile_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_add(int* out, const int* n_dev, long long n_host, const int* tile_sums) {
    const long long n = length(n_dev, n_host);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] += tile_sums[i / kTile];
}

inline int tiles_for(long long n_max) { return (int)((n_max + kTile - 1) / kTile) + 1; }

// out[i] = sum_{j<i} in[i]; *total = sum of all (device).  tile_sums holds
// tiles_for(n_max) ints.  in and out may not alias.
inline cudaError_t exclusive(const int* in, int* out, const int* n_dev, long long n_max, int* tile_sums, int* total,
                             cudaStream_t s) {
    const int ntiles = tiles_for(n_max);
    k_tiles<<<ntiles, kBlock, 0, s>>>(in, n_dev, n_max, out, tile_sums);
    k_sums<<<1, kBlock, 0, s>>>(tile_sums, ntiles, total);
    const long long g = (n_max + 255) / 256;
    k_add<<<(unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g)), 256, 0, s>>>(out, n_dev, n_max, tile_sums);
    return cudaGetLastError();
}

}  // namespace
}  // namespace scan
}  // namespace gtap
