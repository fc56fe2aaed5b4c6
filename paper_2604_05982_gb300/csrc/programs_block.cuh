// Block-mode task programs (Sec. 4.3): every thread of the block runs the
// same step; spawns are per thread; join and completion are block-collective.
#pragma once
#include "gtap_device.cuh"
#include "programs_thread.cuh"

namespace gtap {

// ---------------------------------------------------------------------------
// Mergesort (Cilksort, Sec. 6.3): sort halves in parallel, then merge with a
// forked parallel merge so the top-level merge has no sequential tail.
// Ranges of <= leaf keys are sorted by one block; merges are split along the
// merge path into pieces of <= merge_cutoff output keys, one block each.
//
// Root environment: gtap_mergesort_args.  Records:
//   MSORT  [16] root, into_tmp  [24] lo  [32] hi
//   MMERGE [16] root, flags (bit0: source is tmp, bit1: destination is tmp)
//          [24] a_lo [32] a_hi [40] b_lo [48] b_hi [56] out_lo
struct MsortSpawn { uint32_t root, into_tmp; unsigned long long lo, hi; };
struct MmergeSpawn { uint32_t root, flags; unsigned long long a_lo, a_hi, b_lo, b_hi, out_lo; };

constexpr int kMsTile = 4096;       // output keys merged per shared-memory tile (BS * 16)
constexpr int kMsMaxLeaf = 4096;    // keys sorted in shared memory by one block

__device__ __forceinline__ const gtap_mergesort_args& msort_env(const KParams& P, uint32_t root) {
    return *reinterpret_cast<const gtap_mergesort_args*>(P.root_desc[root].env);
}
__device__ __forceinline__ uint32_t* msort_buf(const gtap_mergesort_args& e, bool tmp) { return tmp ? e.tmp : e.dst; }

// Merge-path split: how many of A's elements precede output position d when
// merging A (na) and B (nb), equal keys taken from A first.
template <class Load>
__device__ __forceinline__ unsigned long long merge_path(unsigned long long na, unsigned long long nb,
                                                         unsigned long long d, Load ld) {
    unsigned long long lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
    while (lo < hi) {
        unsigned long long mid = (lo + hi) >> 1;
        if (ld(true, mid) <= ld(false, d - 1 - mid)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Shared-memory index with one pad word per 32, so that a warp accessing
// element t*ITEMS + k (a stride of ITEMS words) touches 32 different banks.
__device__ __forceinline__ int padx(int i) { return i + (i >> 5); }
constexpr int kMsPadded = kMsTile + kMsTile / 32;
// a tile buffer plus room for the merge windows' reads past the tile's last key
constexpr int kMsStride = kMsPadded + 32;

// Merge path inside shared memory (padded layout): how many of A's elements
// precede output position d; equal keys come from A first.
// The same split found by G lanes together (G divides 32, the group is G
// consecutive lanes of one warp, all active): every round the lanes test G
// evenly spaced candidates at once and the group keeps the gap between the
// last candidate where A still precedes and the first where it does not, so a
// range of n candidates takes about log_{G+1}(n) dependent loads instead of
// log_2(n).  Every lane of the group returns the split.
template <int G, class Load>
__device__ __forceinline__ unsigned long long merge_path_group(unsigned long long na, unsigned long long nb,
                                                               unsigned long long d, Load ld) {
    const int lane = threadIdx.x & 31;
    const int g = lane % G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - g));
    unsigned long long lo = d > nb ? d - nb : 0, hi = d < na ? d : na;   // answer in [lo, hi]
    while (hi - lo > (unsigned long long)G) {
        const unsigned long long span = hi - lo;
        const unsigned long long pos = lo + span * (unsigned long long)(g + 1) / (unsigned long long)(G + 1);
        const bool before = ld(true, pos) <= ld(false, d - 1 - pos);     // answer > pos
        const unsigned m = __ballot_sync(gmask, before) >> (lane - g);
        const int t = __popc(m & ((G == 32) ? 0xffffffffu : ((1u << G) - 1u)));
        // candidates 0..t-1 precede: the answer lies after candidate t-1 and at or before candidate t
        const unsigned long long nlo = (t > 0) ? lo + span * (unsigned long long)t / (unsigned long long)(G + 1) + 1 : lo;
        const unsigned long long nhi = (t < G) ? lo + span * (unsigned long long)(t + 1) / (unsigned long long)(G + 1) : hi;
        lo = nlo;
        hi = nhi;
    }
    // at most G candidates left: test lo + g for g < hi - lo
    const unsigned long long pos = lo + (unsigned long long)g;
    const bool before = pos < hi && ld(true, pos) <= ld(false, d - 1 - pos);
    const unsigned m = __ballot_sync(gmask, before) >> (lane - g);
    return lo + (unsigned long long)__popc(m & ((G == 32) ? 0xffffffffu : ((1u << G) - 1u)));
}

__device__ __forceinline__ int smem_merge_path(const uint32_t* sa, int na, const uint32_t* sb, int nb, int d,
                                               int a0, int b0) {
    int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sa[padx(a0 + mid)] <= sb[padx(b0 + d - 1 - mid)]) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ITEMS consecutive keys of a padded shared-memory run starting at index
// `base`; positions at or past `valid` read as 0xFFFFFFFF.  The window crosses
// at most one 32-word pad boundary, found once.  Reads may go up to
// ITEMS - 1 words past the run (the callers' buffers leave room for that).
template <int ITEMS>
__device__ __forceinline__ void smem_window(const uint32_t* s, int base, int valid, uint32_t (&w)[ITEMS]) {
    const uint32_t* p = s + base + (base >> 5);
    const int cross = 32 - (base & 31);   // first window offset past the next pad word
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const uint32_t x = p[k + (k >= cross ? 1 : 0)];
        w[k] = (k < valid) ? x : 0xFFFFFFFFu;
    }
}

// The N smallest of two ascending sequences a and b, ascending, into a.  The
// element-wise minimum of a and reversed b holds exactly the N smallest of the
// 2N keys and is bitonic (Batcher's bitonic merge, first half-cleaner); the
// remaining half-cleaners sort it.  Only key values are produced, so which of
// two equal keys is taken does not matter.
template <int N>
__device__ __forceinline__ void lowest_of_two_sorted(uint32_t (&a)[N], const uint32_t (&b)[N]) {
#pragma unroll
    for (int k = 0; k < N; ++k) a[k] = min(a[k], b[N - 1 - k]);
#pragma unroll
    for (int j = N / 2; j > 0; j >>= 1) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if ((k & j) == 0) {
                const uint32_t x = a[k], y = a[k + j];
                a[k] = min(x, y);
                a[k + j] = max(x, y);
            }
        }
    }
}

// The ITEMS outputs of merge-path position d of the runs A = s[a0, a0 + na)
// and B = s[b0, b0 + nb) (padded indices), i of them taken from A: the lowest
// ITEMS keys of the windows A[i, i + ITEMS) and B[d - i, d - i + ITEMS).
template <int ITEMS>
__device__ __forceinline__ void smem_window_merge(const uint32_t* s, int a0, int na, int b0, int nb, int i, int d,
                                                  uint32_t (&out)[ITEMS]) {
    uint32_t w[ITEMS];
    smem_window<ITEMS>(s, a0 + i, na - i, out);
    smem_window<ITEMS>(s, b0 + (d - i), nb - (d - i), w);
    lowest_of_two_sorted<ITEMS>(out, w);
}

// Sort of n <= 4096 keys by one block: every thread sorts kItems keys in
// registers with a bitonic network, then log2(BS) rounds of merging pairs of
// sorted runs in shared memory, each thread producing kItems outputs of a
// merge located by a merge-path search.
template <int ITEMS>
__device__ __forceinline__ void sort_registers(uint32_t (&x)[ITEMS]) {
#pragma unroll
    for (int k = 2; k <= ITEMS; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const uint32_t a = x[i], b = x[l];
                    if ((a > b) == up) { x[i] = b; x[l] = a; }
                }
            }
        }
    }
}

template <int BS>
__device__ void block_sort_leaf(const uint32_t* src, int n, uint32_t* dst, uint32_t* sh) {
    constexpr int kItems = kMsMaxLeaf / BS;
    const int t = threadIdx.x;
    for (int i = t; i < kMsMaxLeaf; i += BS) sh[padx(i)] = (i < n) ? __ldg(src + i) : 0xFFFFFFFFu;
    __syncthreads();
    uint32_t x[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) x[k] = sh[padx(t * kItems + k)];
    sort_registers<kItems>(x);
    for (int run = kItems; run < kMsMaxLeaf; run <<= 1) {
        // while a merged pair of runs lies inside one warp's 32 * kItems keys, the
        // warp reads and writes only its own keys: a warp barrier is enough
        const bool warp_local = 2 * run <= 32 * kItems;
        if (warp_local) __syncwarp(); else __syncthreads();
#pragma unroll
        for (int k = 0; k < kItems; ++k) sh[padx(t * kItems + k)] = x[k];
        if (warp_local) __syncwarp(); else __syncthreads();
        const int o = t * kItems;
        const int base = o & ~(2 * run - 1);
        const int d = o - base;
        const int i = smem_merge_path(sh, run, sh, run, d, base, base + run);
        smem_window_merge<kItems>(sh, base, run, base + run, run, i, d, x);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kItems; ++k) sh[padx(t * kItems + k)] = x[k];
    __syncthreads();
    for (int i = t; i < n; i += BS) dst[i] = sh[padx(i)];
    __syncthreads();
}

// Fork the merge of X[a_lo,a_hi) and X[b_lo,b_hi) into Y[out_lo..] as up to
// BS pieces split on the merge path (one search per piece boundary, in parallel).
template <int BS>
__device__ void msort_fork_merge(BTaskCtx& c, const gtap_mergesort_args& e, uint32_t root, uint32_t flags,
                                 unsigned long long a_lo, unsigned long long a_hi, unsigned long long b_lo,
                                 unsigned long long b_hi, unsigned long long out_lo) {
    unsigned long long* split = c.prog_smem<unsigned long long>();
    const unsigned long long na = a_hi - a_lo, nb = b_hi - b_lo, total = na + nb;
    const unsigned long long cut = e.merge_cutoff;
    unsigned long long pieces = (total + cut - 1) / cut;
    if (pieces > (unsigned long long)BS) pieces = BS;
    const uint32_t* X = msort_buf(e, flags & 1u);
    const uint32_t* A = X + a_lo;
    const uint32_t* B = X + b_lo;
    for (int p = threadIdx.x; p <= (int)pieces; p += BS) {
        const unsigned long long d = total * (unsigned long long)p / pieces;
        split[p] = merge_path(na, nb, d, [&](bool inA, unsigned long long k) { return __ldcg((inA ? A : B) + k); });
    }
    __syncthreads();
    if (threadIdx.x < (int)pieces) {
        const int p = threadIdx.x;
        const unsigned long long d0 = total * (unsigned long long)p / pieces, d1 = total * (unsigned long long)(p + 1) / pieces;
        const unsigned long long i0 = split[p], i1 = split[p + 1];
        c.spawn(T_MMERGE, 0,
                MmergeSpawn{root, flags, a_lo + i0, a_lo + i1, b_lo + (d0 - i0), b_lo + (d1 - i1), out_lo + d0});
    }
    __syncthreads();
}

// Asynchronous 4-byte global -> shared copy (cp.async, cached in L1 on the way);
// completion is tracked per thread by commit groups.
__device__ __forceinline__ void cp_async4(uint32_t* sdst, const uint32_t* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

constexpr int kMsStages = 3;   // shared-memory tiles of a merge piece in flight (one merged, the rest loading)

// Merge one piece directly (<= merge_cutoff output keys), tile by tile.
template <int BS>
__device__ void msort_merge_piece(BTaskCtx& c, const gtap_mergesort_args& e, uint32_t flags, unsigned long long a_lo,
                                  unsigned long long a_hi, unsigned long long b_lo, unsigned long long b_hi,
                                  unsigned long long out_lo) {
    uint32_t* sh = c.prog_smem<uint32_t>();
    unsigned long long* split = reinterpret_cast<unsigned long long*>(sh + kMsStages * kMsStride);
    const uint32_t* X = msort_buf(e, flags & 1u);
    uint32_t* Y = msort_buf(e, flags & 2u);
    const unsigned long long na = a_hi - a_lo, nb = b_hi - b_lo, total = na + nb;
    const int tiles = (int)((total + kMsTile - 1) / kMsTile);
    const uint32_t* A = X + a_lo;
    const uint32_t* B = X + b_lo;
    if (tiles > 1) {
        // tile boundaries: 8 lanes per boundary, BS/8 boundaries per round
        constexpr int kG = 8;
        for (int p0 = 0; p0 <= tiles; p0 += BS / kG) {
            const int p = p0 + (int)threadIdx.x / kG;
            const unsigned long long d = min(total, (unsigned long long)min(p, tiles) * kMsTile);
            const unsigned long long sp =
                merge_path_group<kG>(na, nb, d, [&](bool inA, unsigned long long k) { return __ldcg((inA ? A : B) + k); });
            if (p <= tiles && (threadIdx.x % kG) == 0) split[p] = sp;
        }
    } else if (threadIdx.x == 0) {
        split[0] = 0;
        split[1] = na;
    }
    __syncthreads();
    // Pipeline over the piece's tiles: a ring of kMsStages shared-memory tiles
    // filled by cp.async; tile k + kMsStages - 1 is requested while tile k is
    // merged, and merged keys go straight from registers to global memory.
    // One barrier per tile: after it every thread's copies of tile k are
    // visible and every thread has finished merging tile k - 1, whose buffer
    // the newly requested tile reuses.
    constexpr int kItems = kMsTile / BS;
    const int t = threadIdx.x;
    auto tile_bounds = [&](int k, int& tna, int& tnb, unsigned long long& i0, unsigned long long& j0) {
        const unsigned long long d0 = (unsigned long long)k * kMsTile, d1 = min(total, d0 + kMsTile);
        i0 = split[k];
        const unsigned long long i1 = split[k + 1];
        j0 = d0 - i0;
        tna = (int)(i1 - i0);
        tnb = (int)((d1 - i1) - j0);
    };
    auto issue_tile = [&](int k) {   // element t + r*BS of the tile's input (A part, then B part)
        if (k < tiles) {
            int tna, tnb;
            unsigned long long i0, j0;
            tile_bounds(k, tna, tnb, i0, j0);
            uint32_t* dstb = sh + (k % kMsStages) * kMsStride;
            const uint32_t* ga = A + i0;
            const uint32_t* gb = B + j0 - tna;
#pragma unroll
            for (int r = 0; r < kItems; ++r) {
                const int el = t + r * BS;
                if (el < tna + tnb) cp_async4(dstb + padx(el), (el < tna ? ga : gb) + el);
            }
        }
        cp_async_commit();   // an empty group past the last tile keeps the group count uniform
    };
#pragma unroll
    for (int k = 0; k < kMsStages - 1; ++k) issue_tile(k);
    for (int k = 0; k < tiles; ++k) {
        cp_async_wait<kMsStages - 2>();   // this thread's copies of tile k have landed
        __syncthreads();
        issue_tile(k + kMsStages - 1);
        int tna, tnb;
        unsigned long long i0, j0;
        tile_bounds(k, tna, tnb, i0, j0);
        const uint32_t* cur = sh + (k % kMsStages) * kMsStride;
        const int ttot = tna + tnb;
        const int d0 = min(t * kItems, ttot), d1 = min(d0 + kItems, ttot);
        const int i = smem_merge_path(cur, tna, cur, tnb, d0, 0, tna);
        uint32_t v[kItems];
        smem_window_merge<kItems>(cur, 0, tna, tna, tnb, i, d0, v);
        uint32_t* o = Y + out_lo + (unsigned long long)k * kMsTile + d0;
        if (d1 - d0 == kItems && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
#pragma unroll
            for (int r = 0; r < kItems; r += 4) __stcg(reinterpret_cast<uint4*>(o + r), make_uint4(v[r], v[r + 1], v[r + 2], v[r + 3]));
        } else {
#pragma unroll
            for (int r = 0; r < kItems; ++r)
                if (d0 + r < d1) o[r] = v[r];
        }
    }
    cp_async_wait<0>();
    __syncthreads();   // the buffers are free for the block's next task
}

template <int BS>
__device__ void msort_step(BTaskCtx& c) {
    const MsortSpawn a = c.load<MsortSpawn>();
    const gtap_mergesort_args& e = msort_env(c.P, a.root);
    const unsigned long long n = a.hi - a.lo;
    const unsigned long long mid = a.lo + n / 2;
    const bool into_tmp = a.into_tmp != 0;
    switch (c.pc()) {
    case 0:
        if (n <= e.leaf) {
            block_sort_leaf<BS>(e.src + a.lo, (int)n, msort_buf(e, into_tmp) + a.lo, c.prog_smem<uint32_t>());
            c.ret_void();
            return;
        }
        if (threadIdx.x == 0) {
            c.spawn(T_MSORT, 0, MsortSpawn{a.root, into_tmp ? 0u : 1u, a.lo, mid});
            c.spawn(T_MSORT, 0, MsortSpawn{a.root, into_tmp ? 0u : 1u, mid, a.hi});
        }
        c.join(1);
        return;
    case 1: {
        // halves are in the other buffer; merge them into this task's buffer
        const uint32_t flags = (into_tmp ? 0u : 1u) | (into_tmp ? 2u : 0u);
        if (n <= e.merge_cutoff) {
            msort_merge_piece<BS>(c, e, flags, a.lo, mid, mid, a.hi, a.lo);
            c.ret_void();
        } else {
            msort_fork_merge<BS>(c, e, a.root, flags, a.lo, mid, mid, a.hi, a.lo);
            c.join(2);
        }
        return;
    }
    default:
        c.ret_void();
    }
}

template <int BS>
__device__ void mmerge_step(BTaskCtx& c) {
    const MmergeSpawn a = c.load<MmergeSpawn>();
    const gtap_mergesort_args& e = msort_env(c.P, a.root);
    if (c.pc() == 0) {
        const unsigned long long total = (a.a_hi - a.a_lo) + (a.b_hi - a.b_lo);
        if (total <= e.merge_cutoff) {
            msort_merge_piece<BS>(c, e, a.flags, a.a_lo, a.a_hi, a.b_lo, a.b_hi, a.out_lo);
            c.ret_void();
        } else {
            msort_fork_merge<BS>(c, e, a.root, a.flags, a.a_lo, a.a_hi, a.b_lo, a.b_hi, a.out_lo);
            c.join(1);
        }
    } else {
        c.ret_void();
    }
}

// ---------------------------------------------------------------------------
// Adaptive integration, block mode (Program 1(b)).  block_trap splits [a, b]
// into n trapezoids: thread t sums trapezoids t, t+BS, ... in order, then the
// partial sums are combined by the halving tree s[t] += s[t + s].
// Record: [16] a [24] b [32] eps [40] pad [48] l[BS] [48 + 8 BS] r[BS]
struct IntegBlkSpawn { double a, b, eps, pad; };
template <int BS> __host__ __device__ constexpr uint32_t integ_blk_slot_l() { return 6; }
template <int BS> __host__ __device__ constexpr uint32_t integ_blk_slot_r() { return 6 + BS; }
template <int BS> __host__ __device__ constexpr int integ_blk_record() { return 48 + 16 * BS; }

template <int BS>
__device__ double block_trap(double a, double b, int n, double* red) {
    const int t = threadIdx.x;
    const double h = __ddiv_rn(__dsub_rn(b, a), (double)n);
    double s = 0.0;
    for (int i = t; i < n; i += BS) {
        const double x0 = __dadd_rn(a, __dmul_rn(h, (double)i));
        const double x1 = (i + 1 == n) ? b : __dadd_rn(a, __dmul_rn(h, (double)(i + 1)));
        s = __dadd_rn(s, __dmul_rn(__dmul_rn(__dsub_rn(x1, x0), __dadd_rn(runge_fn(x0), runge_fn(x1))), 0.5));
    }
    red[t] = s;
    __syncthreads();
    for (int stride = BS / 2; stride >= 1; stride >>= 1) {
        if (t < stride) red[t] = __dadd_rn(red[t], red[t + stride]);
        __syncthreads();
    }
    const double v = red[0];
    __syncthreads();
    return v;
}

template <int BS>
__device__ void integrate_blk_step(BTaskCtx& c) {
    double* red = c.prog_smem<double>();
    const IntegBlkSpawn s = c.load<IntegBlkSpawn>();
    const int t = threadIdx.x;
    if (c.pc() == 0) {
        constexpr int NTRAP = 256;
        const double coarse = block_trap<BS>(s.a, s.b, NTRAP, red);
        const double fine = block_trap<BS>(s.a, s.b, 2 * NTRAP, red);
        if (fabs(__dsub_rn(fine, coarse)) < s.eps) {
            c.ret((unsigned long long)__double_as_longlong(__ddiv_rn(__dsub_rn(__dmul_rn(4.0, fine), coarse), 3.0)));
            return;
        }
        // locals l, r start at 0.0 on every thread; only the spawning thread receives results
        st_cg64(c.frame + 8 * (integ_blk_slot_l<BS>() + t), 0ull);
        st_cg64(c.frame + 8 * (integ_blk_slot_r<BS>() + t), 0ull);
        const double m = __dmul_rn(0.5, __dadd_rn(s.a, s.b));
        if (t == 0) {
            c.spawn(T_INTEGRATE_BLK, integ_blk_slot_l<BS>(), IntegBlkSpawn{s.a, m, s.eps, 0.0});
            c.spawn(T_INTEGRATE_BLK, integ_blk_slot_r<BS>(), IntegBlkSpawn{m, s.b, s.eps, 0.0});
        }
        c.join(1);
    } else {
        const double l = __longlong_as_double((long long)ld_cg64(c.frame + 8 * (integ_blk_slot_l<BS>() + t)));
        const double r = __longlong_as_double((long long)ld_cg64(c.frame + 8 * (integ_blk_slot_r<BS>() + t)));
        c.ret((unsigned long long)__double_as_longlong(__dadd_rn(l, r)));
    }
}

}  // namespace gtap
