// Thread-mode task programs written as explicit continuation state machines
// (the lowering Sec. 5.2 describes: locals that cross a join live in the task
// record and a switch on the resume point re-enters the function).
//
// Result slots are addressed as (byte offset in the parent record) / 8.
#pragma once
#include "gtap_device.cuh"

namespace gtap {

// ---------------------------------------------------------------------------
// fib(n) with a task at every call (Sec. 6.3 "Fibonacci").
// record: [16] n, route  [24] l  [32] r
struct FibSpawn { int32_t n; int32_t route; };
constexpr uint32_t kFibSlotL = 3, kFibSlotR = 4;

__device__ __forceinline__ void fib_step(TaskCtx& c) {
    const FibSpawn a = c.load<FibSpawn>();
    // route 1 (DAQ with three queues, Sec. 6.3.2): recursive calls, leaves, continuations
    const int qrec = 0, qleaf = a.route ? 1 : 0, qcont = a.route ? 2 : 0;
    if (c.pc() == 0) {
        if (a.n < 2) { c.ret((unsigned long long)(long long)a.n); return; }
        c.spawn(T_FIB, kFibSlotL, (a.n - 1 >= 2) ? qrec : qleaf, FibSpawn{a.n - 1, a.route});
        c.spawn(T_FIB, kFibSlotR, (a.n - 2 >= 2) ? qrec : qleaf, FibSpawn{a.n - 2, a.route});
        c.join(1, qcont);
    } else {
        const long long l = (long long)ld_cg64(c.frame + 8 * kFibSlotL);
        const long long r = (long long)ld_cg64(c.frame + 8 * kFibSlotR);
        c.ret((unsigned long long)(l + r));
    }
}

// ---------------------------------------------------------------------------
// N-Queens by bitmask backtracking, one task per placed row (Sec. 6.3).
// record: [16] cols, diag_l, diag_r, row|n<<8|route<<16  [32] acc (u64, children add into it)
struct NqSpawn { uint32_t cols, dl, dr, meta; unsigned long long acc; unsigned long long pad; };
constexpr uint32_t kNqSlotAcc = 4;

__device__ __forceinline__ void nqueens_step(TaskCtx& c) {
    if (c.pc() == 0) {
        const uint4 a = ld_obj<uint4>(c.frame + kHdrBytes);
        const int row = (int)(a.w & 0xFF), n = (int)((a.w >> 8) & 0xFF), route = (int)(a.w >> 16);
        if (row == n) { c.ret(1ull); return; }
        const uint32_t full = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
        uint32_t avail = ~(a.x | a.y | a.z) & full;
        if (avail == 0) { c.ret(0ull); return; }
        const uint32_t meta = (uint32_t)(row + 1) | ((uint32_t)n << 8) | ((uint32_t)route << 16);
        const int qchild = route ? (row + 1) : 0;  // DAQ: queue = depth mod n_queues
        while (avail) {
            const uint32_t bit = avail & (0u - avail);
            avail ^= bit;
            NqSpawn s{a.x | bit, (a.y | bit) << 1, (a.z | bit) >> 1, meta, 0ull, 0ull};
            c.spawn(T_NQUEENS, kNqSlotAcc, qchild, s, kFlagAccumulate);
        }
        c.join(1, route ? row : 0);
    } else {
        c.ret(ld_cg64(c.frame + 8 * kNqSlotAcc));
    }
}

// ---------------------------------------------------------------------------
// Unbalanced hashed tree.  SplitMix64 (Steele, Lea, Flood 2014): advance the
// state by the golden-ratio increment, then apply the xor-shift-multiply
// finaliser.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long uts_child_id(unsigned long long p, uint32_t i) {
    return splitmix64(p ^ (0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1)));
}
__device__ __forceinline__ uint32_t uts_arity(unsigned long long v, uint32_t m, unsigned long long thr) {
    return splitmix64(v ^ 0xD1B54A32D192ED03ull) < thr ? m : 0u;
}
// A node's result packs (nodes << 32 | leaves) of its subtree; sums of packed
// values add both fields as long as each stays below 2^32.
constexpr unsigned long long kUtsNode = 1ull << 32;

// record: [16] id  [24] threshold  [32] m|route<<8  [36] arity (0xFFFFFFFF: compute)  [40] acc
struct UtsSpawn { unsigned long long id, thr; uint32_t m_route, arity; unsigned long long acc; };
constexpr uint32_t kUtsSlotAcc = 5;
// range record: [16] parent id  [24] threshold  [32] m|route<<8  [36] lo  [40] hi  [44] pad  [48] acc
struct UtsRangeSpawn { unsigned long long id, thr; uint32_t m_route, lo, hi, pad; unsigned long long acc; };
constexpr uint32_t kUtsRangeSlotAcc = 6;
constexpr int kUtsFan = 8;   // children staged per step; wider nodes fork range tasks

__device__ __forceinline__ int uts_child_queue(unsigned long long cid, uint32_t m, unsigned long long thr, int route) {
    if (!route) return 0;
    return uts_arity(cid, m, thr) ? 0 : 1;  // nodes with children -> q0, leaves -> q1
}

// Spawn children [lo, hi) of node `id`: directly when few, else as range tasks.
__device__ __forceinline__ void uts_spawn_children(TaskCtx& c, unsigned long long id, unsigned long long thr,
                                                   uint32_t m_route, uint32_t lo, uint32_t hi, uint32_t slot) {
    const uint32_t m = m_route & 0xFF;
    const int route = (int)((m_route >> 8) & 0xFF);
    const uint32_t n = hi - lo;
    if (n <= (uint32_t)kUtsFan) {
        for (uint32_t i = lo; i < hi; ++i) {
            const unsigned long long cid = uts_child_id(id, i);
            c.spawn(T_UTS, slot, uts_child_queue(cid, m, thr, route), UtsSpawn{cid, thr, m_route, 0xFFFFFFFFu, 0ull},
                    kFlagAccumulate);
        }
    } else {
        const uint32_t per = (n + kUtsFan - 1) / kUtsFan;
        for (uint32_t s = lo; s < hi; s += per) {
            const uint32_t e = min(hi, s + per);
            c.spawn(T_UTS_RANGE, slot, 0, UtsRangeSpawn{id, thr, m_route, s, e, 0u, 0ull}, kFlagAccumulate);
        }
    }
}

// The root record carries the seed and flag kUtsHashRoot: its id is splitmix64(seed).
constexpr uint32_t kUtsHashRoot = 1u << 16;

__device__ __forceinline__ void uts_step(TaskCtx& c) {
    const UtsSpawn a = c.load<UtsSpawn>();
    const int route = (int)((a.m_route >> 8) & 0xFF);
    if (c.pc() == 0) {
        unsigned long long id = a.id;
        uint32_t mr = a.m_route;
        if (mr & kUtsHashRoot) { id = splitmix64(id); mr &= 0xFFFFu; }
        const uint32_t arity = (a.arity != 0xFFFFFFFFu) ? a.arity : uts_arity(id, mr & 0xFF, a.thr);
        if (arity == 0) { c.ret(kUtsNode | 1ull); return; }
        uts_spawn_children(c, id, a.thr, mr, 0, arity, kUtsSlotAcc);
        c.join(1, route ? 2 : 0);
    } else {
        c.ret(a.acc + kUtsNode);
    }
}

__device__ __forceinline__ void uts_range_step(TaskCtx& c) {
    const UtsRangeSpawn a = c.load<UtsRangeSpawn>();
    if (c.pc() == 0) {
        uts_spawn_children(c, a.id, a.thr, a.m_route, a.lo, a.hi, kUtsRangeSlotAcc);
        c.join(1, (a.m_route >> 8) ? 2 : 0);
    } else {
        c.ret(a.acc);
    }
}

// ---------------------------------------------------------------------------
// Adaptive trapezoid integration, thread mode (Program 1(a)).  Explicitly
// rounded double operations (no contraction into fused multiply-add), so the
// result is the same bit pattern as a plain IEEE evaluation on the host.
__device__ __forceinline__ double runge_fn(double x) {
    return __ddiv_rn(1.0, __dadd_rn(1.0, __dmul_rn(__dmul_rn(25.0, x), x)));
}
__device__ __forceinline__ double trap_rn(double a, double b) {
    return __dmul_rn(__dmul_rn(__dsub_rn(b, a), __dadd_rn(runge_fn(a), runge_fn(b))), 0.5);
}
// record: [16] a  [24] b  [32] eps  [40] l  [48] r
struct IntegSpawn { double a, b, eps; double pad; };
constexpr uint32_t kIntSlotL = 5, kIntSlotR = 6;

__device__ __forceinline__ void integrate_step(TaskCtx& c) {
    if (c.pc() == 0) {
        const IntegSpawn s = ld_obj<IntegSpawn>(c.frame + kHdrBytes);
        const double m = __dmul_rn(0.5, __dadd_rn(s.a, s.b));
        const double coarse = trap_rn(s.a, s.b);
        const double fine = __dadd_rn(trap_rn(s.a, m), trap_rn(m, s.b));
        if (fabs(__dsub_rn(fine, coarse)) < s.eps) {
            const double v = __ddiv_rn(__dsub_rn(__dmul_rn(4.0, fine), coarse), 3.0);
            c.ret((unsigned long long)__double_as_longlong(v));
            return;
        }
        c.spawn(T_INTEGRATE, kIntSlotL, 0, IntegSpawn{s.a, m, s.eps, 0.0});
        c.spawn(T_INTEGRATE, kIntSlotR, 0, IntegSpawn{m, s.b, s.eps, 0.0});
        c.join(1, 0);
    } else {
        const double l = __longlong_as_double((long long)ld_cg64(c.frame + 8 * kIntSlotL));
        const double r = __longlong_as_double((long long)ld_cg64(c.frame + 8 * kIntSlotR));
        c.ret((unsigned long long)__double_as_longlong(__dadd_rn(l, r)));
    }
}

}  // namespace gtap
