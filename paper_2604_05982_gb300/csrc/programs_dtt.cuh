// Dual-tree traversal of the Laplace FMM as block-mode tasks (Sec. 6.4.1):
// starting from the root-root pair, every cell pair either passes the MAC
// (appended to the M2L list), is a pair of leaves (appended to the P2P list),
// or is split -- the larger cell, both when the levels are equal, so a self
// pair (A, A) yields all child pairs -- and its child pairs are examined in
// turn.  Lists are fixed-capacity arrays appended with atomicAdd; an append
// beyond the capacity is counted but not stored, so the host sees the size
// it needs (the paper checks capacities on every run).
//
// A task carries up to kDttGroup unresolved pairs.  The block expands its
// frontier in rounds: every pair's child pairs become items (<= 64 per pair),
// one thread per item applies the MAC and the leaf test, and the block
// appends its M2L and P2P entries with one global atomic per list per round.
// Unresolved children form the next frontier; while it holds at most
// kDttLocal pairs the block keeps going in place, otherwise it forks the
// frontier as child tasks of kDttGroup pairs each and joins them (the
// traversal's recursion, with the task granularity set by the frontier).
#pragma once
#include "fmm_internal.h"
#include "gtap_device.cuh"

namespace gtap {

constexpr int kDttLocal = 16;
constexpr int kDttFront = 64 * kDttLocal;
constexpr int kDttMaxSpawn = (kDttFront + fmm::kDttGroup - 1) / fmm::kDttGroup;
static_assert(kDttFront < (1 << 16), "per-round counts are packed in 16-bit fields");

struct DttShared {
    unsigned long long fr[kDttFront];   // frontier of unresolved pairs (target << 32 | source)
    int pstart[kDttLocal + 1];          // first item of each frontier pair
    int pa[kDttLocal], pb[kDttLocal];   // first target / source cell of the pair's children
    int na[kDttLocal], nb[kDttLocal];   // number of them (1 when that side is not split)
    unsigned long long wsum[32];        // per-warp packed counts
    unsigned long long base[2];         // list positions granted to this round
    int misc[4];                        // [0] items this round
};

// MAC with every operation rounded separately, as the oracle evaluates it:
// accept iff (h_A sqrt3 + h_B sqrt3)^2 < theta^2 |c_A - c_B|^2.
__device__ __forceinline__ bool dtt_mac(const fmm::Dbl4& A, const fmm::Dbl4& B, double theta) {
    const double dx = __dsub_rn(A.x, B.x), dy = __dsub_rn(A.y, B.y), dz = __dsub_rn(A.z, B.z);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double R = __dadd_rn(__dmul_rn(A.w, fmm::kSqrt3), __dmul_rn(B.w, fmm::kSqrt3));
    return __dmul_rn(R, R) < __dmul_rn(__dmul_rn(theta, theta), d2);
}

__device__ __forceinline__ fmm::Dbl4 ldg_geom(const fmm::Dbl4* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return fmm::make_dbl4(a.x, a.y, b.x, b.y);
}

template <int BS>
__device__ void dtt_step(BTaskCtx& c) {
    if (c.pc() == 1) {   // resumed after the forked frontier completed
        c.ret_void();
        return;
    }
    constexpr int kPer = kDttFront / BS;
    DttShared& S = *reinterpret_cast<DttShared*>((reinterpret_cast<uintptr_t>(c.bs.prog) + 15) & ~uintptr_t(15));
    const fmm::DttSpawn arg = c.load<fmm::DttSpawn>();
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    // a record that does not describe a traversal task is reported, never followed
    if (arg.root >= c.P.n_roots || arg.n < 1 || arg.n > (uint32_t)fmm::kDttGroup) {
        if (t == 0) c.fail(GTAP_ERR_TASK_FAILED, ((unsigned long long)arg.root << 32) | arg.n);
        c.ret_void();
        return;
    }
    const fmm::DttEnv env = ld_obj_ro<fmm::DttEnv>(c.P.root_desc[arg.root].env);   // immutable during the run
    const fmm::DttAux ax = ld_obj_ro<fmm::DttAux>(env.aux);
    const uint32_t ncell = (uint32_t)env.n_cells;
    int F = (int)arg.n;
    if (t < F) S.fr[t] = arg.pr[t];
    __syncthreads();
    for (;;) {
        // how each frontier pair splits
        if (t < F) {
            const unsigned long long pr = S.fr[t];
            int A = (int)(pr >> 32), B = (int)(pr & 0xFFFFFFFFull);
            if ((uint32_t)A >= ncell || (uint32_t)B >= ncell) {
                c.fail(GTAP_ERR_TASK_FAILED, pr);
                A = B = 0;
            }
            const int4 ia = __ldg(&env.info[A]), ib = __ldg(&env.info[B]);
            const bool la = ia.z < 0, lb = ib.z < 0;
            const int lva = ia.w >> 8, lvb = ib.w >> 8;
            const bool sa = !la && (lb || lva <= lvb);
            const bool sb = !lb && (la || lvb <= lva);
            S.pa[t] = sa ? ia.z : A;
            S.na[t] = sa ? (ia.w & 0xFF) : 1;
            S.pb[t] = sb ? ib.z : B;
            S.nb[t] = sb ? (ib.w & 0xFF) : 1;
        }
        __syncthreads();
        if (t == 0) {
            int s = 0;
            for (int k = 0; k < F; ++k) { S.pstart[k] = s; s += S.na[k] * S.nb[k]; }
            S.pstart[F] = s;
            S.misc[0] = s;
        }
        __syncthreads();
        const int I = S.misc[0];
        // classify the child pairs: 0 = M2L, 1 = P2P, 2 = unresolved, 3 = none.
        // Items are strided over the threads (a round of ~100 items is one item
        // per thread, not 8 dependent items on each of 13 threads while the block
        // waits at the next barrier); lists and frontier take any order.
        unsigned long long iv[kPer];
        int cls[kPer];
        unsigned long long packed = 0;   // three 16-bit counts: M2L, P2P, unresolved
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int i = r * BS + t;
            cls[r] = 3;
            iv[r] = 0;
            if (i < I) {
                int k = 0;
                while (S.pstart[k + 1] <= i) ++k;
                const int j = i - S.pstart[k];
                const int nbk = max(S.nb[k], 1);
                int ca = S.pa[k] + j / nbk, cb = S.pb[k] + j % nbk;
                if ((uint32_t)ca >= ncell || (uint32_t)cb >= ncell) {
                    c.fail(GTAP_ERR_TASK_FAILED, ((unsigned long long)(uint32_t)ca << 32) | (uint32_t)cb);
                    ca = cb = 0;
                }
                iv[r] = ((unsigned long long)(uint32_t)ca << 32) | (uint32_t)cb;
                bool accept = false;
                if (ca != cb) {
                    int decided = 0;   // 1 accept, -1 reject, 0 undecided
                    if (ax.screen) {
                        const int4 la = __ldg(env.lat + ca), lb = __ldg(env.lat + cb);
                        const float dx = (float)(la.x - lb.x), dy = (float)(la.y - lb.y), dz = (float)(la.z - lb.z);
                        const float d2 = dx * dx + dy * dy + dz * dz;
                        const float sh = (float)((1 << (fmm::kMaxLevel - la.w)) + (1 << (fmm::kMaxLevel - lb.w)));
                        const float g = 3.f * sh * sh, f = ax.theta2 * d2;
                        decided = (g < f * (1.f - ax.margin)) ? 1 : (g > f * (1.f + ax.margin)) ? -1 : 0;
                    }
                    accept = decided != 0 ? decided > 0
                                          : dtt_mac(ldg_geom(env.geom + ca), ldg_geom(env.geom + cb), ax.theta);
                }
                if (accept) {
                    cls[r] = 0;
                } else {
                    const int4 ia = __ldg(&env.info[ca]), ib = __ldg(&env.info[cb]);
                    cls[r] = (ia.z < 0 && ib.z < 0) ? 1 : 2;
                }
                packed += 1ull << (16 * cls[r]);
            }
        }
        // block exclusive scan of the packed counts (each field stays <= kDttFront < 2^16)
        unsigned long long incl = packed;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) S.wsum[w] = incl;
        __syncthreads();
        unsigned long long before = 0, total = 0;
        for (int ww = 0; ww < BS / 32; ++ww) {
            const unsigned long long v = S.wsum[ww];
            if (ww < w) before += v;
            total += v;
        }
        const unsigned long long ex = before + incl - packed;
        const int tot0 = (int)(total & 0xFFFFull), tot1 = (int)((total >> 16) & 0xFFFFull),
                  tot2 = (int)((total >> 32) & 0xFFFFull);
        if (t == 0) {
            S.base[0] = tot0 ? atomicAdd(&env.counters[0], (unsigned long long)tot0) : 0ull;
            S.base[1] = tot1 ? atomicAdd(&env.counters[1], (unsigned long long)tot1) : 0ull;
        }
        __syncthreads();
        {
            unsigned long long p0 = S.base[0] + (ex & 0xFFFFull);
            unsigned long long p1 = S.base[1] + ((ex >> 16) & 0xFFFFull);
            int p2 = (int)((ex >> 32) & 0xFFFFull);
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                if (cls[r] == 0) {
                    if (p0 < (unsigned long long)ax.m2l_cap) env.m2l[p0] = iv[r];
                    ++p0;
                } else if (cls[r] == 1) {
                    if (p1 < (unsigned long long)ax.p2p_cap) env.p2p[p1] = iv[r];
                    ++p1;
                } else if (cls[r] == 2) {
                    if (p2 < kDttFront) S.fr[p2] = iv[r];
                    else c.fail(GTAP_ERR_TASK_FAILED, (unsigned long long)p2);
                    ++p2;
                }
            }
        }
        F = min(tot2, kDttFront);
        __syncthreads();
        if (F == 0) {
            c.ret_void();
            return;
        }
        if (F > kDttLocal) {
            const int nch = (F + fmm::kDttGroup - 1) / fmm::kDttGroup;
            if (t < nch) {
                fmm::DttSpawn s;
                s.root = arg.root;
                const int k0 = t * fmm::kDttGroup;
                s.n = (uint32_t)min(fmm::kDttGroup, F - k0);
#pragma unroll
                for (int j = 0; j < fmm::kDttGroup; ++j) s.pr[j] = (j < (int)s.n) ? S.fr[k0 + j] : 0ull;
                c.spawn(T_DTT, 0u, s);
            }
            c.join(1);
            return;
        }
    }
}

}  // namespace gtap
