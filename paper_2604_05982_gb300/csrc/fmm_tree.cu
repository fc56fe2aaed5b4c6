// Adaptive octree construction for the Laplace FMM (Sec. 6.4.1), as plain
// data-parallel kernels around the task-parallel traversal:
//   1. bounding cube of the points (min/max reduction);
//   2. 63-bit Morton codes, 21 bits per axis, q = min(2^21-1, floor((x-lo)*2^21/side));
//   3. stable LSD radix sort of (code, input index), 8 passes of 8 bits, so
//      equal codes keep input order;
//   4. level-synchronous refinement: a cell of level l with more than
//      leaf_size points (and l < 21) splits into its non-empty octants, found
//      by binary search in the sorted codes; child cells are numbered breadth
//      first by a scan of the per-cell child counts.  Level sizes stay on the
//      device, so all 21 levels are enqueued without a host round trip;
//   5. gather of the points into Morton order.
// The geometry is computed in FP64 with every operation rounded separately
// (no contraction), so cell centres and codes are reproducible bit for bit.
#include <cuda_runtime.h>

#include "fmm_internal.h"
#include "scan.cuh"

namespace gtap {
namespace fmm {
namespace {

constexpr int kRsBlock = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsBlock * kRsItems;

__global__ void k_bbox_partial(const double* pos, long long n, double* part) {
    __shared__ double sh[6][256];
    double mn[3] = {pos[0], pos[1], pos[2]}, mx[3] = {pos[0], pos[1], pos[2]};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        for (int d = 0; d < 3; ++d) {
            const double v = pos[3 * i + d];
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
    for (int d = 0; d < 3; ++d) { sh[d][threadIdx.x] = mn[d]; sh[3 + d][threadIdx.x] = mx[d]; }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int d = 0; d < 3; ++d) {
                sh[d][threadIdx.x] = fmin(sh[d][threadIdx.x], sh[d][threadIdx.x + o]);
                sh[3 + d][threadIdx.x] = fmax(sh[3 + d][threadIdx.x], sh[3 + d][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

// box = {lo x, lo y, lo z, side, scale}; root cell written here too.
__global__ void k_bbox_final(const double* part, int nparts, long long n, double* box, Dbl4* geom, int4* info,
                             int4* lat, int* lstart, int* flags) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double mn[3], mx[3];
    for (int d = 0; d < 3; ++d) { mn[d] = part[d]; mx[d] = part[3 + d]; }
    for (int b = 1; b < nparts; ++b)
        for (int d = 0; d < 3; ++d) { mn[d] = fmin(mn[d], part[6 * b + d]); mx[d] = fmax(mx[d], part[6 * b + 3 + d]); }
    double side = 0.0;
    for (int d = 0; d < 3; ++d) side = fmax(side, __dsub_rn(mx[d], mn[d]));
    if (!(side > 0.0)) side = 1.0;
    const double half = __dmul_rn(side, 0.5);
    double c[3];
    for (int d = 0; d < 3; ++d) {
        const double lo = __dsub_rn(__dmul_rn(__dadd_rn(mn[d], mx[d]), 0.5), half);
        box[d] = lo;
        c[d] = __dadd_rn(lo, half);
    }
    box[3] = side;
    box[4] = __ddiv_rn(2097152.0, side);
    geom[0] = make_dbl4(c[0], c[1], c[2], half);
    info[0] = make_int4(0, (int)n, -1, 0);
    lat[0] = make_int4(1 << 21, 1 << 21, 1 << 21, 0);
    lstart[0] = 0;
    lstart[1] = 1;
    for (int i = 0; i < 4; ++i) flags[i] = 0;
}

__device__ __forceinline__ unsigned long long spread21(unsigned long long v) {
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x1F00000000FFFFull;
    v = (v | (v << 16)) & 0x1F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ unsigned long long compact21(unsigned long long v) {
    v &= 0x1249249249249249ull;
    v = (v | (v >> 2)) & 0x10C30C30C30C30C3ull;
    v = (v | (v >> 4)) & 0x100F00F00F00F00Full;
    v = (v | (v >> 8)) & 0x1F0000FF0000FFull;
    v = (v | (v >> 16)) & 0x1F00000000FFFFull;
    v = (v | (v >> 32)) & 0x1FFFFFull;
    return v;
}

__global__ void k_codes(const double* pos, long long n, const double* box, unsigned long long* keys, uint32_t* vals) {
    const double lo0 = box[0], lo1 = box[1], lo2 = box[2], scale = box[4];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double lo[3] = {lo0, lo1, lo2};
        unsigned long long q[3];
        for (int d = 0; d < 3; ++d) {
            double f = floor(__dmul_rn(__dsub_rn(pos[3 * i + d], lo[d]), scale));
            f = fmin(fmax(f, 0.0), 2097151.0);
            q[d] = (unsigned long long)f;
        }
        keys[i] = spread21(q[0]) | (spread21(q[1]) << 1) | (spread21(q[2]) << 2);
        vals[i] = (uint32_t)i;
    }
}

__global__ void __launch_bounds__(kRsBlock) k_rs_hist(const unsigned long long* keys, long long n, int shift, int* hist,
                                                      int ntiles) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRsTile;
    for (int k = 0; k < kRsItems; ++k) {
        const long long i = base + k * kRsBlock + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255ull], 1);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: within a tile, items keep their order per digit (warp match
// gives the rank inside a warp, per-warp digit counts order the warps).
__global__ void __launch_bounds__(kRsBlock) k_rs_scatter(const unsigned long long* kin, const uint32_t* vin,
                                                         unsigned long long* kout, uint32_t* vout, long long n,
                                                         int shift, const int* offs, int ntiles) {
    __shared__ int base[256];
    __shared__ int wc[kRsBlock / 32][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    base[t] = offs[t * ntiles + blockIdx.x];
    const long long tile = (long long)blockIdx.x * kRsTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int k = 0; k < kRsItems; ++k) {
#pragma unroll
        for (int ww = 0; ww < kRsBlock / 32; ++ww) wc[ww][t] = 0;
        __syncthreads();
        const long long i = tile + k * kRsBlock + t;
        const bool valid = i < n;
        unsigned long long key = 0;
        uint32_t val = 0;
        int d = 256 + lane;               // unique per invalid lane: never grouped
        if (valid) { key = kin[i]; val = vin[i]; d = (int)((key >> shift) & 255ull); }
        const unsigned m = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(m & lt);
        if (valid && rank == 0) wc[w][d] = __popc(m);
        __syncthreads();
        if (valid) {
            int pos = base[d] + rank;
            for (int ww = 0; ww < w; ++ww) pos += wc[ww][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        int add = 0;
#pragma unroll
        for (int ww = 0; ww < kRsBlock / 32; ++ww) add += wc[ww][t];
        base[t] += add;
        __syncthreads();
    }
}

// Level l: child counts of every cell (octant boundaries by binary search).
__global__ void k_level_count(int l, const unsigned long long* codes, const int4* info, const int* lstart, int leaf,
                              int* bounds, int* cnt, int* lvl_n) {
    const int lo = lstart[l], hi = lstart[l + 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) lvl_n[l] = hi - lo;
    const int shift = 3 * (20 - l);
    for (int c = lo + blockIdx.x * blockDim.x + threadIdx.x; c < hi; c += gridDim.x * blockDim.x) {
        const int4 in = info[c];
        int nch = 0;
        if (in.y > leaf && l < kMaxLevel) {
            const int first = in.x, end = in.x + in.y;
            int* bd = bounds + 9 * (size_t)(c - lo);
            bd[0] = first;
            bd[8] = end;
            for (int o = 1; o < 8; ++o) {
                int a = first, b = end;   // first k with octant >= o
                while (a < b) {
                    const int mid = (a + b) >> 1;
                    if ((int)((codes[mid] >> shift) & 7ull) < o) a = mid + 1; else b = mid;
                }
                bd[o] = a;
            }
            for (int o = 0; o < 8; ++o) nch += (bd[o + 1] > bd[o]) ? 1 : 0;
        }
        cnt[c - lo] = nch;
    }
}

__global__ void k_level_write(int l, const unsigned long long* codes, int4* info, Dbl4* geom, int4* lat, int* lstart,
                              const double* box, const int* bounds, const int* cnt, const int* off,
                              const int* lvl_total, int cap, int* flags) {
    const int lo = lstart[l], hi = lstart[l + 1];
    const int next = hi + lvl_total[l];
    if (blockIdx.x == 0 && threadIdx.x == 0) lstart[l + 2] = (next <= cap) ? next : hi;
    if (next > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) flags[0] = 1;
        return;
    }
    const double side = box[3];
    const int cl = l + 1;
    const double cell = __ddiv_rn(side, (double)(1ull << cl));
    const double half = __dmul_rn(cell, 0.5);
    const int cshift = 3 * (21 - cl);
    for (int c = lo + blockIdx.x * blockDim.x + threadIdx.x; c < hi; c += gridDim.x * blockDim.x) {
        const int nch = cnt[c - lo];
        if (nch == 0) continue;
        const int cf = hi + off[c - lo];
        int4 in = info[c];
        in.z = cf;
        in.w = (l << 8) | nch;
        info[c] = in;
        const int* bd = bounds + 9 * (size_t)(c - lo);
        int j = 0;
        for (int o = 0; o < 8; ++o) {
            const int s = bd[o], e = bd[o + 1];
            if (e <= s) continue;
            const unsigned long long pre = codes[s] >> cshift;
            const unsigned long long jx = compact21(pre), jy = compact21(pre >> 1), jz = compact21(pre >> 2);
            const double ix = (double)jx, iy = (double)jy, iz = (double)jz;
            const int sh = kMaxLevel - cl;
            lat[cf + j] = make_int4((int)((2 * jx + 1) << sh), (int)((2 * jy + 1) << sh), (int)((2 * jz + 1) << sh), cl);
            geom[cf + j] = make_dbl4(__dadd_rn(box[0], __dmul_rn(__dadd_rn(ix, 0.5), cell)),
                                        __dadd_rn(box[1], __dmul_rn(__dadd_rn(iy, 0.5), cell)),
                                        __dadd_rn(box[2], __dmul_rn(__dadd_rn(iz, 0.5), cell)), half);
            info[cf + j] = make_int4(s, e - s, -1, cl << 8);
            ++j;
        }
    }
}

__global__ void k_gather(const double* pos, const double* q, const uint32_t* order, long long n, Dbl4* pts) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const uint32_t i = order[k];
        pts[k] = make_dbl4(pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2], q[i]);
    }
}

// One warp per cell: leaf points relative to the leaf centre, in FP32.
__global__ void k_leaf_local(const Dbl4* pts, const Dbl4* geom, const int4* info, int n_cells, float4* ploc) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((long long)gridDim.x * blockDim.x) >> 5);
    for (int c = warp; c < n_cells; c += nw) {
        const int4 in = info[c];
        if (in.z >= 0) continue;
        const Dbl4 g = geom[c];
        for (int k = in.x + lane; k < in.x + in.y; k += 32) {
            const Dbl4 p = pts[k];
            ploc[k] = make_float4((float)(p.x - g.x), (float)(p.y - g.y), (float)(p.z - g.z), (float)p.w);
        }
    }
}

int grid_for(long long n, int block, int cap) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

int radix_tiles(long long n) { return (int)((n + kRsTile - 1) / kRsTile); }

// Levels from `from` down are empty (the refinement stopped early): their
// start entries all equal lstart[from], as the full level loop would leave them.
__global__ void k_lstart_tail(int* lstart, int from) {
    const int v = lstart[from];
    for (int k = from + 1 + (int)threadIdx.x; k <= kMaxLevel + 1; k += blockDim.x) lstart[k] = v;
}

// Structural check of the cell records before any kernel follows their links:
// flags[1] = 1 on a malformed record; flags[2] = leaves; flags[3] = largest leaf.
// The cell count is read from lstart[kMaxLevel + 1], never above `cap`.
__global__ void k_check_tree(const int4* info, const int* lstart, int cap, long long n, int* flags) {
    const int n_cells = min(lstart[kMaxLevel + 1], cap);
    int bad = 0, leaves = 0, big = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_cells; i += gridDim.x * blockDim.x) {
        const int4 c = info[i];
        const int level = c.w >> 8, nch = c.w & 0xFF;
        bool ok = c.x >= 0 && c.y >= 1 && (long long)c.x + c.y <= n && level >= 0 && level <= kMaxLevel;
        if (c.z >= 0) {
            ok = ok && c.z > i && nch >= 1 && nch <= 8 && (long long)c.z + nch <= n_cells;
            if (ok)
                for (int j = 0; j < nch; ++j) ok = ok && (info[c.z + j].w >> 8) == level + 1;
        } else {
            ok = ok && c.z == -1 && nch == 0;
            if (ok) {
                ++leaves;
                big = max(big, c.y);
            }
        }
        if (!ok) bad = 1;
    }
    bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
    leaves = (int)__reduce_add_sync(0xffffffffu, (unsigned)leaves);
    big = (int)__reduce_max_sync(0xffffffffu, (unsigned)big);
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(&flags[1], 1);
        if (leaves) atomicAdd(&flags[2], leaves);
        if (big) atomicMax(&flags[3], big);
    }
}

cudaError_t launch_tree_sort(TreeBufs& b, cudaStream_t s) {
    const long long n = b.n;
    k_bbox_partial<<<kBoxParts, 256, 0, s>>>(b.pos, n, b.bbox_part);
    k_bbox_final<<<1, 32, 0, s>>>(b.bbox_part, kBoxParts, n, b.box, b.geom, b.info, b.lat, b.lstart, b.flags);
    k_codes<<<grid_for(n, 256, 4096), 256, 0, s>>>(b.pos, n, b.box, b.keys[0], b.vals[0]);
    const int ntiles = radix_tiles(n);
    int cur = 0;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        k_rs_hist<<<ntiles, kRsBlock, 0, s>>>(b.keys[cur], n, shift, b.hist, ntiles);
        cudaError_t e = scan::exclusive(b.hist, b.hist_scan, nullptr, 256LL * ntiles, b.tile_sums, nullptr, s);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<ntiles, kRsBlock, 0, s>>>(b.keys[cur], b.vals[cur], b.keys[cur ^ 1], b.vals[cur ^ 1], n, shift,
                                                 b.hist_scan, ntiles);
        cur ^= 1;
    }
    b.codes = b.keys[cur];
    b.order = b.vals[cur];
    return cudaGetLastError();
}

cudaError_t launch_tree_levels(const TreeBufs& b, int l0, int l1, cudaStream_t s) {
    const int g = grid_for(b.cap_cells, 256, 1216);
    for (int l = l0; l < l1 && l < kMaxLevel; ++l) {
        k_level_count<<<g, 256, 0, s>>>(l, b.codes, b.info, b.lstart, b.leaf, b.bounds, b.cnt, b.lvl_n);
        cudaError_t e = scan::exclusive(b.cnt, b.off, b.lvl_n + l, b.cap_cells, b.tile_sums, b.lvl_total + l, s);
        if (e != cudaSuccess) return e;
        k_level_write<<<g, 256, 0, s>>>(l, b.codes, b.info, b.geom, b.lat, b.lstart, b.box, b.bounds, b.cnt, b.off,
                                        b.lvl_total, b.cap_cells, b.flags);
    }
    return cudaGetLastError();
}

cudaError_t launch_tree_finish(const TreeBufs& b, int levels_done, cudaStream_t s) {
    if (levels_done < kMaxLevel) k_lstart_tail<<<1, 32, 0, s>>>(b.lstart, levels_done + 1);
    k_gather<<<grid_for(b.n, 256, 4096), 256, 0, s>>>(b.pos, b.q, b.order, b.n, b.pts);
    k_check_tree<<<grid_for(b.cap_cells, 256, 1216), 256, 0, s>>>(b.info, b.lstart, b.cap_cells, b.n, b.flags);
    return cudaGetLastError();
}

cudaError_t launch_leaf_local(const TreeBufs& b, int n_cells, cudaStream_t s) {
    k_leaf_local<<<grid_for((long long)n_cells * 32, 256, 4096), 256, 0, s>>>(b.pts, b.geom, b.info, n_cells, b.ploc);
    return cudaGetLastError();
}

}  // namespace fmm
}  // namespace gtap
