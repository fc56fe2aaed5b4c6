// Execution-mode and DAQ microbenchmark programs (Sec. 6.1 "Understanding
// the Execution Modes", Sec. 6.2 "Effect of Divergence-Aware Queueing"): a
// full binary task tree of depth D whose leaves each run the same
// data-parallel compute loop of `iters` iterations.  With K > 1 each leaf runs
// one of K equal-cost compute functions with distinct control flow, chosen by
// a hash of the node id, so it is known when the leaf is spawned and DAQ can
// route leaves of one function to one queue.
//
// Definitions (shared with the public header's gtap_bintree_args):
//   node ids: root 1, children of v are 2v and 2v+1, leaves are the nodes of
//   level D;  leaf function k(v) = (splitmix64(v) >> 32) mod K (0 if K == 1);
//   leaf value = sum over i in [0, iters) of g_k((v << 32) + i), mod 2^64;
//   the tree's result is the sum of its leaf values, mod 2^64.
#pragma once
#include "gtap_device.cuh"
#include "programs_thread.cuh"

namespace gtap {

__device__ __forceinline__ unsigned long long bt_rotl(unsigned long long z, int r) { return (z << r) | (z >> (64 - r)); }

// The four compute functions: a multiply-xorshift mix, an xorshift-multiply,
// an add-multiply-rotate and an xorshift-multiply-xorshift.  Each costs two
// 64-bit multiplies or one multiply and a rotate, plus a few shifts and xors;
// their instruction sequences differ, so lanes running different ones diverge.
__device__ __forceinline__ unsigned long long bt_g0(unsigned long long x) {
    unsigned long long z = x * 0x9E3779B97F4A7C15ull;
    z ^= z >> 29;
    z *= 0xBF58476D1CE4E5B9ull;
    return z ^ (z >> 32);
}
__device__ __forceinline__ unsigned long long bt_g1(unsigned long long x) {
    unsigned long long z = x ^ (x << 13);
    z ^= z >> 7;
    z ^= z << 17;
    return z * 0x2545F4914F6CDD1Dull;
}
__device__ __forceinline__ unsigned long long bt_g2(unsigned long long x) {
    unsigned long long z = (x + 0x632BE59BD9B4E019ull) * 0x94D049BB133111EBull;
    return bt_rotl(z, 23) ^ (z >> 11);
}
__device__ __forceinline__ unsigned long long bt_g3(unsigned long long x) {
    unsigned long long z = x ^ (x >> 32);
    z *= 0xD6E8FEB86659FD93ull;
    return z ^ (z >> 28);
}

__device__ __forceinline__ int bt_leaf_fn(unsigned long long id, int K) {
    return K > 1 ? (int)((splitmix64(id) >> 32) % (unsigned long long)K) : 0;
}

// Iterations [i0, iters) with stride `step` of leaf `id`'s loop under function k.
__device__ __forceinline__ unsigned long long bt_loop(unsigned long long id, int k, int i0, int iters, int step) {
    const unsigned long long base = id << 32;
    unsigned long long acc = 0;
    switch (k) {
    case 0: for (int i = i0; i < iters; i += step) acc += bt_g0(base + (unsigned)i); break;
    case 1: for (int i = i0; i < iters; i += step) acc += bt_g1(base + (unsigned)i); break;
    case 2: for (int i = i0; i < iters; i += step) acc += bt_g2(base + (unsigned)i); break;
    default: for (int i = i0; i < iters; i += step) acc += bt_g3(base + (unsigned)i); break;
    }
    return acc;
}

// Record payload (both modes): [16] id  [24] level, depth  [32] iters, K | route << 8 | cutoff << 16
struct BtSpawn { unsigned long long id; uint32_t level, depth; uint32_t iters, kr; };
constexpr int kBtMaxK = 4;

// ---------------------------------------------------------------------------
// Thread mode: one lane runs a leaf's whole loop.  Children add their value
// into the parent's accumulator (record word 5).
struct BtThreadSpawn { unsigned long long id; uint32_t level, depth; uint32_t iters, kr; unsigned long long acc; };
constexpr uint32_t kBtSlotAcc = 5;

__device__ __forceinline__ void bintree_step(TaskCtx& c) {
    const BtThreadSpawn a = c.load<BtThreadSpawn>();
    const int K = (int)(a.kr & 0xFF), route = (int)((a.kr >> 8) & 0xFF);
    if (c.pc() != 0) { c.ret(a.acc); return; }
    if (a.level == a.depth) {
        c.ret(bt_loop(a.id, bt_leaf_fn(a.id, K), 0, (int)a.iters, 1));
        return;
    }
    // DAQ routing (route 1): inner nodes and continuations -> queue 0, a leaf of
    // compute function k -> queue 1 + k
    const bool leaves = a.level + 1 == a.depth;
#pragma unroll
    for (uint32_t b = 0; b < 2; ++b) {
        const unsigned long long cid = 2 * a.id + b;
        const int q = (route && leaves) ? 1 + bt_leaf_fn(cid, K) : 0;
        c.spawn(T_BINTREE, kBtSlotAcc, q, BtThreadSpawn{cid, a.level + 1, a.depth, a.iters, a.kr, 0ull}, kFlagAccumulate);
    }
    c.join(1, 0);
}

// ---------------------------------------------------------------------------
// Block mode: the block runs a leaf's loop data-parallel (iterations strided
// over the threads, then a block reduction).  With a cutoff c > 0, a node c
// levels above the leaves runs its whole subtree (2^c leaves) as one task, the
// coarsening Sec. 6.1 applies to recover thread mode's batching.  Child values
// arrive in record words 5 (left, spawned by thread 0) and 6 (right, thread 1).
constexpr uint32_t kBtBlkSlot = 5;

template <int BS>
__device__ __forceinline__ unsigned long long bt_block_sum(unsigned long long v, unsigned long long* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long s = 0;
#pragma unroll
    for (int w = 0; w < BS / 32; ++w) s += red[w];
    __syncthreads();
    return s;   // every thread holds the block's sum
}

template <int BS>
__device__ void bintree_blk_step(BTaskCtx& c) {
    unsigned long long* red = c.prog_smem<unsigned long long>();
    const BtSpawn a = c.load<BtSpawn>();
    const int K = (int)(a.kr & 0xFF), cutoff = (int)((a.kr >> 16) & 0xFF);
    const int t = threadIdx.x;
    if (c.pc() != 0) {
        const unsigned long long l = ld_cg64(c.frame + 8 * kBtBlkSlot);
        const unsigned long long r = ld_cg64(c.frame + 8 * (kBtBlkSlot + 1));
        c.ret(l + r);
        return;
    }
    const int below = (int)(a.depth - a.level);
    if (below == 0 || (cutoff > 0 && below <= cutoff)) {
        // leaves 2^below consecutive ids starting at id << below
        const unsigned long long first = a.id << below;
        const int nleaves = 1 << below;
        const int iters = (int)a.iters;
        unsigned long long acc = 0;
        if (iters >= BS || nleaves == 1) {
            for (int l = 0; l < nleaves; ++l) {
                const unsigned long long id = first + (unsigned)l;
                acc += bt_loop(id, bt_leaf_fn(id, K), t, iters, BS);
            }
        } else {
            // few iterations per leaf: spread (leaf, iteration) pairs over the threads
            const long long total = (long long)nleaves * iters;
            for (long long f = t; f < total; f += BS) {
                const unsigned long long id = first + (unsigned long long)(f / iters);
                const int i = (int)(f % iters);
                acc += bt_loop(id, bt_leaf_fn(id, K), i, i + 1, 1);
            }
        }
        c.ret(bt_block_sum<BS>(acc, red));
        return;
    }
    if (t < 2)
        c.spawn(T_BINTREE_BLK, kBtBlkSlot, BtSpawn{2 * a.id + (unsigned)t, a.level + 1, a.depth, a.iters, a.kr});
    c.join(1);
}

}  // namespace gtap
