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

// One block merges A[0,na) and B[0,nb) (na + nb <= BS * 16) into out, via shared memory.
template <int BS>
__device__ void block_merge_tile(const uint32_t* A, int na, const uint32_t* B, int nb, uint32_t* out, uint32_t* sh) {
    constexpr int kItems = kMsTile / BS;
    uint32_t* shin = sh;
    uint32_t* shout = sh + kMsTile;
    const int t = threadIdx.x;
    for (int i = t; i < na; i += BS) shin[i] = __ldcg(A + i);
    for (int i = t; i < nb; i += BS) shin[na + i] = __ldcg(B + i);
    __syncthreads();
    const int total = na + nb;
    const int d0 = min(t * kItems, total), d1 = min(d0 + kItems, total);
    int lo = d0 > nb ? d0 - nb : 0, hi = d0 < na ? d0 : na;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (shin[mid] <= shin[na + d0 - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    int i = lo, j = d0 - lo;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (d0 + k < d1) {
            const bool takeA = (j >= nb) || (i < na && shin[i] <= shin[na + j]);
            shout[d0 + k] = takeA ? shin[i++] : shin[na + j++];
        }
    }
    __syncthreads();
    for (int k = t; k < total; k += BS) out[k] = shout[k];
    __syncthreads();
}

// Bitonic sort of n <= 4096 keys in shared memory (padded to a power of two).
template <int BS>
__device__ void block_sort_leaf(const uint32_t* src, int n, uint32_t* dst, uint32_t* sh) {
    const int t = threadIdx.x;
    int np = 1;
    while (np < n) np <<= 1;
    for (int i = t; i < np; i += BS) sh[i] = (i < n) ? __ldg(src + i) : 0xFFFFFFFFu;
    __syncthreads();
    for (int k = 2; k <= np; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = t; p < (np >> 1); p += BS) {
                const int i = 2 * j * (p / j) + (p % j);
                const int q = i + j;
                const uint32_t a = sh[i], b = sh[q];
                const bool up = (i & k) == 0;
                if ((a > b) == up) { sh[i] = b; sh[q] = a; }
            }
            __syncthreads();
        }
    }
    for (int i = t; i < n; i += BS) dst[i] = sh[i];
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

// Merge one piece directly (<= merge_cutoff output keys), tile by tile.
template <int BS>
__device__ void msort_merge_piece(BTaskCtx& c, const gtap_mergesort_args& e, uint32_t flags, unsigned long long a_lo,
                                  unsigned long long a_hi, unsigned long long b_lo, unsigned long long b_hi,
                                  unsigned long long out_lo) {
    uint32_t* sh = c.prog_smem<uint32_t>();
    unsigned long long* split = reinterpret_cast<unsigned long long*>(sh + 2 * kMsTile);
    const uint32_t* X = msort_buf(e, flags & 1u);
    uint32_t* Y = msort_buf(e, flags & 2u);
    const unsigned long long na = a_hi - a_lo, nb = b_hi - b_lo, total = na + nb;
    const int tiles = (int)((total + kMsTile - 1) / kMsTile);
    const uint32_t* A = X + a_lo;
    const uint32_t* B = X + b_lo;
    if (tiles > 1) {
        for (int p = threadIdx.x; p <= tiles; p += BS) {
            const unsigned long long d = min(total, (unsigned long long)p * kMsTile);
            split[p] = merge_path(na, nb, d, [&](bool inA, unsigned long long k) { return __ldcg((inA ? A : B) + k); });
        }
    } else if (threadIdx.x == 0) {
        split[0] = 0;
        split[1] = na;
    }
    __syncthreads();
    for (int k = 0; k < tiles; ++k) {
        const unsigned long long d0 = (unsigned long long)k * kMsTile, d1 = min(total, d0 + kMsTile);
        const unsigned long long i0 = split[k], i1 = split[k + 1];
        block_merge_tile<BS>(A + i0, (int)(i1 - i0), B + (d0 - i0), (int)((d1 - i1) - (d0 - i0)), Y + out_lo + d0, sh);
    }
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
