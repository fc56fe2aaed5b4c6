// Thread-mode task programs written as explicit continuation state machines
// (the lowering Sec. 5.2 describes: locals that cross a join live in the task
// record and a switch on the resume point re-enters the function).
//
// Result slots are addressed as (byte offset in the parent record) / 8.
#pragma once
#include "gtap_device.cuh"

namespace gtap {

// ---------------------------------------------------------------------------
// fib(n) with a task at every call (Sec. 6.3 "Fibonacci"), or with a
// sequential cutoff (Sec. 6.3.2): a call with n below the cutoff is a leaf
// task that computes fib(n) by the serial recursion inside its lane.
// record: [16] n, route | cutoff << 8  [24] l  [32] r
struct FibSpawn { int32_t n; int32_t rc; };
constexpr uint32_t kFibSlotL = 3, kFibSlotR = 4;

// The serial recursion fib(n) = fib(n-1) + fib(n-2) with an explicit stack of
// pending calls (n < 64, so at most n + 1 entries).
static __device__ __noinline__ long long fib_serial(int n) {
    int stack[64];
    int sp = 0;
    long long acc = 0;
    stack[sp++] = n;
    while (sp > 0) {
        const int m = stack[--sp];
        if (m < 2) { acc += m; continue; }
        stack[sp++] = m - 1;
        stack[sp++] = m - 2;
    }
    return acc;
}

__device__ __forceinline__ void fib_step(TaskCtx& c) {
    const FibSpawn a = c.load<FibSpawn>();
    const int route = a.rc & 0xFF, cutoff = a.rc >> 8;
    // route 1 (DAQ with three queues, Sec. 6.3.2): recursive calls, leaves, continuations
    const int qrec = 0, qleaf = route ? 1 : 0, qcont = route ? 2 : 0;
    if (c.pc() == 0) {
        if (a.n < 2 || a.n < cutoff) { c.ret((unsigned long long)fib_serial(a.n)); return; }
        const int n1 = a.n - 1, n2 = a.n - 2;
        c.spawn(T_FIB, kFibSlotL, (n1 >= 2 && n1 >= cutoff) ? qrec : qleaf, FibSpawn{n1, a.rc});
        c.spawn(T_FIB, kFibSlotR, (n2 >= 2 && n2 >= cutoff) ? qrec : qleaf, FibSpawn{n2, a.rc});
        c.join(1, qcont);
    } else {
        const long long l = (long long)c.word<kFibSlotL>();
        const long long r = (long long)c.word<kFibSlotR>();
        c.ret((unsigned long long)(l + r));
    }
}

// ---------------------------------------------------------------------------
// N-Queens by bitmask backtracking, one task per placed row (Sec. 6.3), or
// with a cutoff depth (Sec. 6.3.1): a board with `depth` rows placed is a leaf
// task that finishes the search serially in its lane.
// record: [16] cols, diag_l, diag_r, row | n << 8 | route << 16 | depth << 24  [32] acc (u64, children add into it)
struct NqSpawn { uint32_t cols, dl, dr, meta; unsigned long long acc; unsigned long long pad; };
constexpr uint32_t kNqSlotAcc = 4;

// Serial backtracking from a partial board: one (cols, dl, dr, remaining
// candidates) frame per placed row, at most 16 rows.
static __device__ __noinline__ unsigned long long nq_serial(int n, int row, uint32_t cols, uint32_t dl, uint32_t dr) {
    if (row == n) return 1ull;
    const uint32_t full = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
    uint32_t sc[17], sl[17], sr[17], sa[17];
    int top = 0;
    sc[0] = cols; sl[0] = dl; sr[0] = dr; sa[0] = ~(cols | dl | dr) & full;
    unsigned long long sols = 0;
    const int rows_left = n - row;
    while (top >= 0) {
        const uint32_t avail = sa[top];
        if (avail == 0) { --top; continue; }
        const uint32_t bit = avail & (0u - avail);
        sa[top] = avail ^ bit;
        if (top + 1 == rows_left) { ++sols; continue; }
        const uint32_t c2 = sc[top] | bit, l2 = (sl[top] | bit) << 1, r2 = (sr[top] | bit) >> 1;
        ++top;
        sc[top] = c2; sl[top] = l2; sr[top] = r2; sa[top] = ~(c2 | l2 | r2) & full;
    }
    return sols;
}

__device__ __forceinline__ void nqueens_step(TaskCtx& c) {
    if (c.pc() == 0) {
        const uint4 a = c.load<uint4>();
        const int row = (int)(a.w & 0xFF), n = (int)((a.w >> 8) & 0xFF), route = (int)((a.w >> 16) & 0xFF);
        const int depth = (int)(a.w >> 24);
        if (row == n) { c.ret(1ull); return; }
        if (depth > 0 && row >= depth) { c.ret(nq_serial(n, row, a.x, a.y, a.z)); return; }
        const uint32_t full = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
        uint32_t avail = ~(a.x | a.y | a.z) & full;
        if (avail == 0) { c.ret(0ull); return; }
        const uint32_t meta = (uint32_t)(row + 1) | (a.w & 0xFFFFFF00u);
        // DAQ: route 1 = queue depth mod n_queues; route 2 = recursive tasks q0, cutoff leaves q1
        const int qchild = route == 1 ? (row + 1) : (route == 2 ? ((depth > 0 && row + 1 >= depth) ? 1 : 0) : 0);
        while (avail) {
            const uint32_t bit = avail & (0u - avail);
            avail ^= bit;
            NqSpawn s{a.x | bit, (a.y | bit) << 1, (a.z | bit) >> 1, meta, 0ull, 0ull};
            c.spawn(T_NQUEENS, kNqSlotAcc, qchild, s, kFlagAccumulate);
        }
        c.join(1, route == 1 ? row : 0);
    } else {
        c.ret(c.word<kNqSlotAcc>());
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
        const IntegSpawn s = c.load<IntegSpawn>();
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
        const double l = __longlong_as_double((long long)c.word<kIntSlotL>());
        const double r = __longlong_as_double((long long)c.word<kIntSlotR>());
        c.ret((unsigned long long)__double_as_longlong(__dadd_rn(l, r)));
    }
}

}  // namespace gtap

namespace gtap {

// ---------------------------------------------------------------------------
// k-clique counting by orientation (Sec. 6.4.2).  For a DAG edge (u, v),
// C = N+(u) n N+(v); count(S, 1) = |S|, count(S, j) = sum over w in S of
// count(S n N+(w), j - 1).  A set of at most `thr` (<= 64) vertices is counted
// inside the lane with 64-bit adjacency bitsets; a larger one is forked over
// its branch range (the paper's split on the spawn-time estimate |C|).
//
// Sets of the first level, C = N+(u) n N+(v), are spawned unmaterialised:
// the record names P = N+(u), the vertex w = v and |C|, and the child writes C
// to the scratch arena when it first runs.  The edge-range tasks then only
// count, and the expensive intersections are spread over the set tasks that
// idle lanes steal (k = 4, scale 20: 874 -> 769 ms), while waiting first-level
// tasks hold no scratch.  Deeper sets are materialised by the spawning lane:
// that keeps the lanes expanding the frontier busy, and with DAQ choosing the
// fullest queue, cheap unmaterialised spawns at every level let the waiting
// frontier outgrow the frame pool (k = 5, scale 18, 1 GiB pool).
//
// Records (64 bytes):
//   KC range [16] root, lo, hi, pad   [32] acc  [40] local
//   KC set   [16] root, j  [24] set pointer  [32] len, lo  [40] hi, own  [48] acc  [56] local
//   own = kKcLazy: not materialised yet; set/len are P = N+(u), lo is w = v, hi is |C|
//   own = 1: materialised set in a recycled scratch block, freed by this task when its subtree is done
//   own = 0: a branch range of a set owned by an ancestor (or a set in never-recycled scratch)
struct KcRangeSpawn { uint32_t root, lo, hi, pad; unsigned long long acc, local; };
struct KcSetSpawn { uint32_t root, j; unsigned long long set; uint32_t len, lo, hi, own; unsigned long long acc, local; };
constexpr uint32_t kKcRangeSlotAcc = 4, kKcRangeLocal = 40;
constexpr uint32_t kKcSetSlotAcc = 6, kKcSetLocal = 56;
constexpr uint32_t kKcSetPtr = 24, kKcSetLenLo = 32, kKcSetHiOwn = 40;
constexpr uint32_t kKcLazy = 2;
constexpr int kKcFan = 8;          // children per split
constexpr int kKcMaxThr = 64;      // in-lane sets use 64-bit bitsets

// The root environment is immutable during a batch run (read-only path, L1);
// in a served session the poller writes root slots while the kernel runs, so
// it is read through L2 there.
__device__ __forceinline__ gtap_kclique_args kc_env(const KParams& P, uint32_t root) {
    return P.serving ? ld_obj<gtap_kclique_args>(P.root_desc[root].env)
                     : ld_obj_ro<gtap_kclique_args>(P.root_desc[root].env);
}

// Read-only adjacency (never written during a run): non-coherent cached loads.
struct AdjLoad { __device__ int operator()(const int* p) const { return __ldg(p); } };
// Sets in the scratch arena are written during the run: loads through L2.
struct SetLoad { __device__ int operator()(const int* p) const { return __ldcg(p); } };

// |a n b| for sorted lists; the first `cap` common elements go to out (if not null).
template <class LA, class LB>
static __device__ int kc_intersect(const int* a, int na, LA la, const int* b, int nb, LB lb, int* out, int cap) {
    int cnt = 0;
    if (na == 0 || nb == 0) return 0;
    if ((long long)na * 8 < nb) {
        // gallop the short list's elements through the long one
        int lo = 0;
        for (int i = 0; i < na && lo < nb; ++i) {
            const int x = la(a + i);
            int step = 1, hi = lo;
            while (hi < nb && lb(b + hi) < x) { lo = hi + 1; hi = lo + step; step <<= 1; }
            if (hi > nb) hi = nb;
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (lb(b + mid) < x) lo = mid + 1; else hi = mid; }
            if (lo < nb && lb(b + lo) == x) { if (out && cnt < cap) out[cnt] = x; ++cnt; ++lo; }
        }
    } else if ((long long)nb * 8 < na) {
        int lo = 0;
        for (int i = 0; i < nb && lo < na; ++i) {
            const int x = lb(b + i);
            int step = 1, hi = lo;
            while (hi < na && la(a + hi) < x) { lo = hi + 1; hi = lo + step; step <<= 1; }
            if (hi > na) hi = na;
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (la(a + mid) < x) lo = mid + 1; else hi = mid; }
            if (lo < na && la(a + lo) == x) { if (out && cnt < cap) out[cnt] = x; ++cnt; ++lo; }
        }
    } else {
        // branch-free merge: lanes of a warp with different data take the same path
        // every iteration (only the trip counts differ)
        int i = 0, j = 0;
        while (i < na && j < nb) {
            const int x = la(a + i), y = lb(b + j);
            if (x == y) {
                if (out && cnt < cap) out[cnt] = x;
                ++cnt;
            }
            i += (x <= y) ? 1 : 0;
            j += (y <= x) ? 1 : 0;
        }
    }
    return cnt;
}

static __device__ unsigned long long kc_count_rows(const unsigned long long* row, int ns, int j);

// count(S, j) for |S| <= 64 inside one lane, with 64-bit adjacency bitsets.
static __device__ unsigned long long kc_count_small(const int* S, int ns, int j, const int64_t* off, const int* adj) {
    if (j == 1) return (unsigned long long)ns;
    if (ns < j) return 0;
    unsigned long long row[kKcMaxThr];
    for (int a = 0; a < ns; ++a) {
        // row[a] = members of S that are out-neighbours of S[a]
        const long long b0 = (long long)__ldg(reinterpret_cast<const long long*>(off) + S[a]);
        const int len = (int)((long long)__ldg(reinterpret_cast<const long long*>(off) + S[a] + 1) - b0);
        const int* nb = adj + b0;
        unsigned long long bits = 0;
        if (len > 4 * ns) {
            int lo = 0;
            for (int b = 0; b < ns && lo < len; ++b) {
                const int x = S[b];
                int hi = len;
                while (lo < hi) { const int mid = (lo + hi) >> 1; if (__ldg(nb + mid) < x) lo = mid + 1; else hi = mid; }
                if (lo < len && __ldg(nb + lo) == x) { bits |= 1ull << b; ++lo; }
            }
        } else {
            int i = 0, b = 0;
            while (i < len && b < ns) {   // branch-free merge
                const int x = __ldg(nb + i), y = S[b];
                bits |= (x == y) ? (1ull << b) : 0ull;
                i += (x <= y) ? 1 : 0;
                b += (y <= x) ? 1 : 0;
            }
        }
        row[a] = bits;
    }
    return kc_count_rows(row, ns, j);
}

// count(S, j) from S's adjacency rows (bit b of row[a]: S[b] is an out-neighbour of S[a]), ns <= 64.
static __device__ unsigned long long kc_count_rows(const unsigned long long* row, int ns, int j) {
    if (j == 1) return (unsigned long long)ns;
    if (ns < j) return 0;
    const unsigned long long full = (ns == 64) ? ~0ull : ((1ull << ns) - 1ull);
    if (j == 2) {
        unsigned long long t = 0;
        for (int a = 0; a < ns; ++a) t += (unsigned)__popcll(row[a]);
        return t;
    }
    // depth-first over choices; M = candidates at a level, R = those not yet tried there
    unsigned long long M[16], R[16];
    M[0] = full;
    R[0] = full;
    int l = 0;
    unsigned long long total = 0;
    while (l >= 0) {
        if (R[l] == 0) { --l; continue; }
        const int a = __ffsll((long long)R[l]) - 1;
        R[l] &= R[l] - 1;
        const unsigned long long mn = M[l] & row[a];
        const int rem = j - l - 1;
        if (rem == 1) {
            total += (unsigned)__popcll(mn);
        } else if (rem == 2) {
            for (unsigned long long w = mn; w; w &= w - 1) total += (unsigned)__popcll(mn & row[__ffsll((long long)w) - 1]);
        } else if (__popcll(mn) >= rem) {
            ++l;
            M[l] = mn;
            R[l] = mn;
        }
    }
    return total;
}

// ---------------------------------------------------------------------------
// Pivoting (Sec. 6.4.2, the second k-clique algorithm).  A candidate set of at
// most 64 vertices is encoded as 64-bit adjacency rows: bit b of row a says
// that members a and b are adjacent (in either direction of the DAG).  The
// pivot search counts the cliques of the set that contain exactly r more
// vertices: at a node (S, r still to choose, p pivots) the pivot x is the
// member of S with the most neighbours in S (lowest position on ties); the
// branches are x and the members of S not adjacent to x, in position order;
// branch w recurses on S n N(w) without the earlier branch vertices, w counted
// as a pivot when it is x and as chosen otherwise.  An empty S adds C(p, r);
// r = 0 adds 1 (only the all-pivot path leads to a leaf); a node with fewer
// than r members and pivots together adds nothing.
struct LocalRows { const unsigned long long* r; __device__ unsigned long long operator()(int i) const { return r[i]; } };
struct ScratchRows { const unsigned long long* r; __device__ unsigned long long operator()(int i) const { return __ldcg(r + i); } };

__device__ __forceinline__ unsigned long long kp_binom(int n, int r) {
    if (r < 0 || r > n) return 0ull;
    unsigned long long c = 1;
    for (int i = 1; i <= r; ++i) c = c * (unsigned long long)(n - r + i) / (unsigned long long)i;   // n <= 64, r <= 16
    return c;
}

template <class R>
__device__ __forceinline__ int kp_pivot(R row, unsigned long long S) {
    int best = -1, bx = 0;
    for (unsigned long long t = S; t; t &= t - 1) {
        const int x = __ffsll((long long)t) - 1;
        const int c = __popcll(row(x) & S);
        if (c > best) { best = c; bx = x; }
    }
    return bx;
}

constexpr int kKpStack = 66;   // every child set is smaller than its parent's: depth <= 64 + 1

template <class R>
static __device__ __noinline__ unsigned long long kp_count(R row, unsigned long long S0, int r0, int p0) {
    unsigned long long st_s[kKpStack], st_rem[kKpStack];
    unsigned char st_r[kKpStack], st_p[kKpStack], st_x[kKpStack];
    int top = -1;
    unsigned long long total = 0;
    auto enter = [&](unsigned long long S, int r, int p) {
        if (r < 0) return;
        if (r == 0) { total += 1; return; }
        if (__popcll(S) + p < r) return;
        if (S == 0) { total += kp_binom(p, r); return; }
        const int x = kp_pivot(row, S);
        ++top;
        st_s[top] = S;
        st_rem[top] = S & ~row(x);
        st_r[top] = (unsigned char)r;
        st_p[top] = (unsigned char)p;
        st_x[top] = (unsigned char)x;
    };
    enter(S0, r0, p0);
    while (top >= 0) {
        const unsigned long long rem = st_rem[top];
        if (rem == 0) { --top; continue; }
        const int w = __ffsll((long long)rem) - 1;
        st_rem[top] = rem & (rem - 1);
        const unsigned long long branches = st_s[top] & ~row(st_x[top]);
        const unsigned long long Sw = row(w) & st_s[top] & ~(branches & ((1ull << w) - 1ull));
        if (w == (int)st_x[top]) enter(Sw, st_r[top], st_p[top] + 1);
        else enter(Sw, st_r[top] - 1, st_p[top]);
    }
    return total;
}

// Adjacency rows of the candidate set S[0 .. ns) (ns <= 64, sorted by id), both
// directions: each DAG edge inside S is found from its earlier endpoint's
// out-list, then mirrored.
static __device__ void kp_rows(const int* S, int ns, const int64_t* off, const int* adj, unsigned long long* row) {
    for (int a = 0; a < ns; ++a) {
        const long long b0 = (long long)__ldg(reinterpret_cast<const long long*>(off) + S[a]);
        const int len = (int)((long long)__ldg(reinterpret_cast<const long long*>(off) + S[a] + 1) - b0);
        const int* nb = adj + b0;
        unsigned long long bits = 0;
        int i = 0, b = 0;
        if (len > 4 * ns) {
            int lo = 0;
            for (b = 0; b < ns && lo < len; ++b) {
                const int x = S[b];
                int hi = len;
                while (lo < hi) { const int mid = (lo + hi) >> 1; if (__ldg(nb + mid) < x) lo = mid + 1; else hi = mid; }
                if (lo < len && __ldg(nb + lo) == x) { bits |= 1ull << b; ++lo; }
            }
        } else {
            while (i < len && b < ns) {
                const int x = __ldg(nb + i), y = S[b];
                if (x < y) ++i;
                else if (y < x) ++b;
                else { bits |= 1ull << b; ++i; ++b; }
            }
        }
        row[a] = bits;
    }
    // mirror: adding the mirror of a mirrored bit changes nothing, so one pass in place is enough
    for (int b = 0; b < ns; ++b)
        for (unsigned long long t = row[b]; t; t &= t - 1) row[__ffsll((long long)t) - 1] |= 1ull << b;
}

// r-cliques of the candidate set S[0 .. ns) by the pivot search, in the lane.
static __device__ __noinline__ unsigned long long kp_count_small(const int* S, int ns, int r, const int64_t* off,
                                                                 const int* adj) {
    if (r == 1) return (unsigned long long)ns;
    if (ns < r) return 0;
    unsigned long long row[kKcMaxThr];
    kp_rows(S, ns, off, adj, row);
    const unsigned long long full = (ns == 64) ? ~0ull : ((1ull << ns) - 1ull);
    return kp_count(LocalRows{row}, full, r, 0);
}

// Candidate sets in the scratch arena: a set that fits one block is recycled
// when the set task that owns it is done with it.
__device__ __forceinline__ int* kc_scratch_alloc(TaskCtx& c, int n, bool* pooled) {
    return reinterpret_cast<int*>(scratch_alloc(c.P, (uint64_t)n * 4, pooled, c.type(), c.worker));
}

__device__ __forceinline__ int kc_queue(const gtap_kclique_args& e, int depth) { return e.route ? depth : 0; }
__device__ __forceinline__ long long kc_off(const gtap_kclique_args& e, long long v) {
    return __ldg(reinterpret_cast<const long long*>(e.off) + v);
}

// Bitset-encoded split (Sec. 6.4.2, pivoting): a candidate set too heavy for
// one lane (more than split_threshold members, at most 64) is encoded as its
// adjacency rows in a recycled scratch block, and a task over its pivot's
// branch range is forked; that task splits the range over child tasks (each
// re-applies the test) or runs its branches itself.
// Record: [16] root  [20] r:8 | p:8 | lo:8 | hi:8  [24] rows  [32] S  [40] branches (0: not chosen yet)
//         [48] x:8 | own:8 | depth:8  [56] acc
struct KpSpawn { uint32_t root, meta; unsigned long long rows, S, vp; uint32_t xo, pad; unsigned long long acc; };
constexpr uint32_t kKpSlotAcc = 7;
constexpr uint32_t kKpRows = 24, kKpBranches = 40, kKpXo = 48;

__device__ __forceinline__ bool kp_spawn_split(TaskCtx& c, const gtap_kclique_args& e, uint32_t root, const int* S,
                                               int ns, int r, int depth, uint32_t slot) {
    unsigned long long row[kKcMaxThr];
    kp_rows(S, ns, e.off, e.adj, row);
    bool pooled;
    unsigned long long* blk = reinterpret_cast<unsigned long long*>(scratch_alloc(c.P, (uint64_t)ns * 8, &pooled, c.type(), c.worker));
    if (!blk) return false;
    for (int a = 0; a < ns; ++a) __stcg(blk + a, row[a]);
    const unsigned long long full = (ns == 64) ? ~0ull : ((1ull << ns) - 1ull);
    c.spawn(T_KCLIQUE_PIV, slot, kc_queue(e, depth),
            KpSpawn{root, (uint32_t)r | (255u << 24), (unsigned long long)blk, full, 0ull,
                    (pooled ? 1u : 0u) << 8 | ((uint32_t)depth << 16), 0u, 0ull},
            kFlagAccumulate);
    return true;
}

static __device__ void kclique_piv_step(TaskCtx& c) {
    const KpSpawn a = c.load<KpSpawn>();
    const unsigned long long* rows = reinterpret_cast<const unsigned long long*>(a.rows);
    const bool own = ((a.xo >> 8) & 0xFF) != 0;
    if (c.pc() != 0) {
        if (own) scratch_free(c.P, rows, c.type(), c.worker);
        c.ret(a.acc);
        return;
    }
    const gtap_kclique_args e = kc_env(c.P, a.root);
    const ScratchRows row{rows};
    const int r = (int)(a.meta & 0xFF), p = (int)((a.meta >> 8) & 0xFF);
    const int depth = (int)((a.xo >> 16) & 0xFF);
    unsigned long long vp = a.vp;
    int x = (int)(a.xo & 0xFF);
    if (vp == 0) {
        // first run on this set: choose the pivot; the branches are x and its non-neighbours
        x = kp_pivot(row, a.S);
        vp = a.S & ~row(x);
        st_cg64(c.frame + kKpBranches, vp);
    }
    const int nb = __popcll(vp);
    const int lo = (int)((a.meta >> 16) & 0xFF), hi = min((int)(a.meta >> 24), nb);
    if (hi - lo > kKcFan) {
        const int per = (hi - lo + kKcFan - 1) / kKcFan;
        for (int s0 = lo; s0 < hi; s0 += per)
            c.spawn(T_KCLIQUE_PIV, kKpSlotAcc, kc_queue(e, depth + 1),
                    KpSpawn{a.root, (uint32_t)r | ((uint32_t)p << 8) | ((uint32_t)s0 << 16) | ((uint32_t)min(hi, s0 + per) << 24),
                            a.rows, a.S, vp, (uint32_t)x | ((uint32_t)(depth + 1) << 16), 0u, 0ull},
                    kFlagAccumulate);
        if (own) {
            // the owner frees the rows once its children are done
            st_cg64(c.frame + kKpXo, (unsigned long long)((uint32_t)x | (1u << 8) | ((uint32_t)depth << 16)));
        }
        c.join(1, kc_queue(e, depth));
        return;
    }
    // branches lo .. hi-1 (in bit order) in this lane
    unsigned long long total = 0;
    unsigned long long t = vp;
    for (int i = 0; i < lo; ++i) t &= t - 1;
    for (int i = lo; i < hi; ++i) {
        const int w = __ffsll((long long)t) - 1;
        t &= t - 1;
        const unsigned long long Sw = row(w) & a.S & ~(vp & ((1ull << w) - 1ull));
        total += (w == x) ? kp_count(row, Sw, r, p + 1) : kp_count(row, Sw, r - 1, p);
    }
    if (own) scratch_free(c.P, rows, c.type(), c.worker);
    c.ret(total);
}

// Pivoting on candidate sets of more than 64 vertices (multi-word bitsets).
// The first run of an edge's node materialises C = P n N+(w) and the rows of
// the subgraph C induces (ceil(|C| / 64) words per member, both directions)
// in one scratch allocation; every node keeps its own set S and branch set
// (the pivot and its non-neighbours) in a small block.  A node chooses its
// pivot on its first run; a node with more than kKcFan branches splits the
// branch range over child tasks; otherwise it runs its branches: a branch set
// of at most 64 members is compacted to 64-bit rows and counted in the lane,
// a larger one becomes a child node.
// Record: [16] root  [20] r:8 | p:8 | W:8 | flags:8 (1 lazy, 2 owns rows, 4 owns set, 8 branches chosen,
//         16 rows block pooled, 32 set block pooled)
//         (16/32: the rows / set block is a recycled one-block buffer; 64/128: a recycled large chunk)
//         [24] rows (lazy: P = N+(u))  [32] set block (lazy: w | |P| << 32)
//         [40] lo:16 | hi:16 | x:16 | depth:8 (lazy: |C| in lo/hi)  [48] local  [56] acc
struct KpbSpawn { uint32_t root, meta; unsigned long long rows, set, range, local, acc; };
constexpr uint32_t kKpbSlotAcc = 7;
constexpr uint32_t kKpbMeta = 16, kKpbRows = 24, kKpbSet = 32, kKpbRange = 40, kKpbLocal = 48;
constexpr int kKpbMaxW = 16;   // members up to 1024 (the DAG's out-lists are at most 8192, C is much smaller in practice)
constexpr uint32_t kKpbLazy = 1, kKpbOwnRows = 2, kKpbOwnSet = 4, kKpbChosen = 8, kKpbRowsPooled = 16, kKpbSetPooled = 32,
                   kKpbRowsLarge = 64, kKpbSetLarge = 128;

// Release the blocks a node owns (each block once: a root's set lies inside its rows block).
__device__ __forceinline__ void kpb_release(TaskCtx& c, uint32_t flags, const void* rows, const void* setb) {
    if (flags & kKpbOwnSet) scratch_free_kind(c.P, setb, (flags & kKpbSetPooled) ? 1 : ((flags & kKpbSetLarge) ? 2 : 0),
                                              c.type(), c.worker);
    if (flags & kKpbOwnRows) scratch_free_kind(c.P, rows, (flags & kKpbRowsPooled) ? 1 : ((flags & kKpbRowsLarge) ? 2 : 0),
                                               c.type(), c.worker);
}

__device__ __forceinline__ unsigned long long kpb_range(uint32_t lo, uint32_t hi, uint32_t x, uint32_t depth) {
    return (unsigned long long)(lo & 0xFFFF) | ((unsigned long long)(hi & 0xFFFF) << 16) |
           ((unsigned long long)(x & 0xFFFF) << 32) | ((unsigned long long)(depth & 0xFF) << 48);
}

// A branch set of at most 64 members as a compact 64-bit subgraph, then the pivot count.
__device__ __forceinline__ unsigned long long kpb_count_compact(const unsigned long long* rows, int W,
                                                                 const unsigned long long* Sw, int r, int p) {
    int m[kKcMaxThr];
    int c = 0;
    for (int t = 0; t < W; ++t)
        for (unsigned long long b = Sw[t]; b; b &= b - 1) m[c++] = t * 64 + __ffsll((long long)b) - 1;
    unsigned long long row[kKcMaxThr];
    for (int i = 0; i < c; ++i) {
        const unsigned long long* ri = rows + (size_t)m[i] * W;
        unsigned long long bits = 0;
        for (int j = 0; j < c; ++j)
            if ((__ldcg(ri + (m[j] >> 6)) >> (m[j] & 63)) & 1ull) bits |= 1ull << j;
        row[i] = bits;
    }
    const unsigned long long full = (c == 64) ? ~0ull : ((1ull << c) - 1ull);
    return kp_count(LocalRows{row}, full, r, p);
}

static __device__ void kclique_pivb_step(TaskCtx& c) {
    const KpbSpawn a = c.load<KpbSpawn>();
    uint32_t flags = a.meta >> 24;
    const int r = (int)(a.meta & 0xFF), p = (int)((a.meta >> 8) & 0xFF);
    int W = (int)((a.meta >> 16) & 0xFF);
    if (c.pc() != 0) {
        kpb_release(c, flags, reinterpret_cast<const void*>(a.rows), reinterpret_cast<const void*>(a.set));
        c.ret(a.acc + a.local);
        return;
    }
    const gtap_kclique_args e = kc_env(c.P, a.root);
    unsigned long long* rows = reinterpret_cast<unsigned long long*>(a.rows);
    unsigned long long* setb = reinterpret_cast<unsigned long long*>(a.set);
    uint32_t depth = (uint32_t)((a.range >> 48) & 0xFF);
    uint32_t lo = (uint32_t)(a.range & 0xFFFF), hi = (uint32_t)((a.range >> 16) & 0xFFFF);
    uint32_t x = (uint32_t)((a.range >> 32) & 0xFFFF);
    unsigned long long S[kKpbMaxW], V[kKpbMaxW];
    if (flags & kKpbLazy) {
        // materialise C = P n N+(w) and the rows of the subgraph it induces, in one allocation
        const int* P = reinterpret_cast<const int*>(a.rows);
        const int w = (int)(a.set & 0xFFFFFFFFull), np = (int)(a.set >> 32);
        const int cn = (int)lo;
        W = (cn + 63) / 64;
        if (W > kKpbMaxW) { c.fail(GTAP_ERR_INVALID_ARG, (unsigned long long)cn); return; }
        const uint64_t words = (uint64_t)cn * W + 2 * (uint64_t)W;
        int kind;
        char* blk = scratch_alloc_kind(c.P, words * 8 + (uint64_t)cn * 4, &kind, c.type(), c.worker);
        if (!blk) return;
        rows = reinterpret_cast<unsigned long long*>(blk);
        setb = rows + (size_t)cn * W;
        int* C = reinterpret_cast<int*>(setb + 2 * W);
        const long long ow = kc_off(e, w);
        kc_intersect(P, np, AdjLoad{}, e.adj + ow, (int)(kc_off(e, w + 1) - ow), AdjLoad{}, C, cn);
        for (uint64_t i = 0; i < (uint64_t)cn * W; ++i) __stcg(rows + i, 0ull);
        // DAG edges inside C from each member's out-list, set in both rows
        for (int i = 0; i < cn; ++i) {
            const int y = __ldcg(C + i);
            const long long oy = kc_off(e, y);
            const int ny = (int)(kc_off(e, y + 1) - oy);
            int u0 = 0, v0 = 0;
            while (u0 < ny && v0 < cn) {
                const int s0 = __ldg(e.adj + oy + u0), t0 = __ldcg(C + v0);
                if (s0 < t0) ++u0;
                else if (t0 < s0) ++v0;
                else {
                    unsigned long long* ri = rows + (size_t)i * W + (v0 >> 6);
                    __stcg(ri, __ldcg(ri) | (1ull << (v0 & 63)));
                    unsigned long long* rj = rows + (size_t)v0 * W + (i >> 6);
                    __stcg(rj, __ldcg(rj) | (1ull << (i & 63)));
                    ++u0; ++v0;
                }
            }
        }
        for (int t = 0; t < W; ++t) {
            const int rem_bits = cn - t * 64;
            S[t] = rem_bits >= 64 ? ~0ull : ((1ull << rem_bits) - 1ull);
        }
        // the set block lies inside the rows allocation: freeing the rows frees it (one free per block)
        flags = kKpbOwnRows | (kind == 1 ? kKpbRowsPooled : 0u) | (kind == 2 ? kKpbRowsLarge : 0u);
        lo = 0;
        hi = 0xFFFF;
        // what the resume needs: the blocks to free
        st_cg64(c.frame + kKpbRows, (unsigned long long)rows);
        st_cg64(c.frame + kKpbSet, (unsigned long long)setb);
        st_cg32(c.frame + kKpbMeta, (uint32_t)r | ((uint32_t)p << 8) | ((uint32_t)W << 16) | (flags << 24));
    } else {
        for (int t = 0; t < W; ++t) S[t] = __ldcg(setb + t);
    }
    if (!(flags & kKpbChosen)) {
        // the pivot: most neighbours inside S, lowest position on ties; the branches: x and its non-neighbours
        int best = -1;
        for (int t = 0; t < W; ++t)
            for (unsigned long long b = S[t]; b; b &= b - 1) {
                const int y = t * 64 + __ffsll((long long)b) - 1;
                int cnt = 0;
                for (int q = 0; q < W; ++q) cnt += __popcll(__ldcg(rows + (size_t)y * W + q) & S[q]);
                if (cnt > best) { best = cnt; x = (uint32_t)y; }
            }
        for (int t = 0; t < W; ++t) {
            V[t] = S[t] & ~__ldcg(rows + (size_t)x * W + t);
            __stcg(setb + W + t, V[t]);
        }
        flags |= kKpbChosen;
    } else {
        for (int t = 0; t < W; ++t) V[t] = __ldcg(setb + W + t);
    }
    int nb = 0;
    for (int t = 0; t < W; ++t) nb += __popcll(V[t]);
    hi = min(hi, (uint32_t)nb);
    if (hi - lo > (uint32_t)kKcFan) {
        const uint32_t per = (hi - lo + kKcFan - 1) / kKcFan;
        for (uint32_t s0 = lo; s0 < hi; s0 += per)
            c.spawn(T_KCLIQUE_PIVB, kKpbSlotAcc, kc_queue(e, (int)depth + 1),
                    KpbSpawn{a.root, (uint32_t)r | ((uint32_t)p << 8) | ((uint32_t)W << 16) | (kKpbChosen << 24),
                             (unsigned long long)rows, (unsigned long long)setb,
                             kpb_range(s0, min(hi, s0 + per), x, depth + 1), 0ull, 0ull},
                    kFlagAccumulate);
        st_cg32(c.frame + kKpbMeta, (uint32_t)r | ((uint32_t)p << 8) | ((uint32_t)W << 16) | (flags << 24));
        c.join(1, kc_queue(e, (int)depth));
        return;
    }
    // branches lo .. hi-1 of V, in bit order
    unsigned long long local = 0;
    int idx = 0;
    for (int t = 0; t < W && idx < (int)hi; ++t) {
        for (unsigned long long b = V[t]; b && idx < (int)hi; b &= b - 1, ++idx) {
            if (idx < (int)lo) continue;
            const int bit = __ffsll((long long)b) - 1;
            const int w = t * 64 + bit;
            const bool is_x = (uint32_t)w == x;
            const int r2 = is_x ? r : r - 1, p2 = is_x ? p + 1 : p;
            if (r2 < 0) continue;
            if (r2 == 0) { local += 1; continue; }
            // S_w = row(w) n S without the branch vertices before w
            unsigned long long Sw[kKpbMaxW];
            int cnt = 0;
            for (int q = 0; q < W; ++q) {
                const unsigned long long before = q < t ? V[q] : (q == t ? (V[q] & ((1ull << bit) - 1ull)) : 0ull);
                Sw[q] = __ldcg(rows + (size_t)w * W + q) & S[q] & ~before;
                cnt += __popcll(Sw[q]);
            }
            if (cnt + p2 < r2) continue;
            if (cnt == 0) { local += kp_binom(p2, r2); continue; }
            if (cnt <= kKcMaxThr) { local += kpb_count_compact(rows, W, Sw, r2, p2); continue; }
            int kind;
            unsigned long long* nb2 = reinterpret_cast<unsigned long long*>(scratch_alloc_kind(c.P, (uint64_t)W * 16, &kind, c.type(), c.worker));
            if (!nb2) return;
            for (int q = 0; q < W; ++q) __stcg(nb2 + q, Sw[q]);
            c.spawn(T_KCLIQUE_PIVB, kKpbSlotAcc, kc_queue(e, (int)depth + 1),
                    KpbSpawn{a.root, (uint32_t)r2 | ((uint32_t)p2 << 8) | ((uint32_t)W << 16) |
                                         ((kKpbOwnSet | (kind == 1 ? kKpbSetPooled : 0u) | (kind == 2 ? kKpbSetLarge : 0u)) << 24),
                             (unsigned long long)rows, (unsigned long long)nb2, kpb_range(0, 0xFFFF, 0, depth + 1), 0ull, 0ull},
                    kFlagAccumulate);
        }
    }
    if (c.nspawned == 0) {
        kpb_release(c, flags, rows, setb);
        c.ret(local);
        return;
    }
    st_cg64(c.frame + kKpbLocal, local);
    st_cg32(c.frame + kKpbMeta, (uint32_t)r | ((uint32_t)p << 8) | ((uint32_t)W << 16) | (flags << 24));
    c.join(1, kc_queue(e, (int)depth));
}

template <bool SCRATCH>
__device__ __forceinline__ int kc_ld(const int* p) { return SCRATCH ? __ldcg(p) : __ldg(p); }

template <bool SCRATCH>
__device__ __forceinline__ bool kc_contains(const int* L, int n, int x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (kc_ld<SCRATCH>(L + mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo < n && kc_ld<SCRATCH>(L + lo) == x;
}

__device__ __forceinline__ int kc_index_of(const int* C, int n, int x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (C[mid] < x) lo = mid + 1; else hi = mid;
    }
    return (lo < n && C[lo] == x) ? lo : -1;
}

// The lanes of `mask` that run a cooperative pass (see below) and their shared area.
struct KcCoop {
    unsigned mask, below;
    int lane, nact, rank, leader;
    int* cbuf;
    unsigned long long* rows;
    int* claim;
};

// Claims the warp's area for the lanes now converged here; false when another
// group of the same warp holds it.
__device__ __forceinline__ bool kc_coop_begin(KcCoop& k, int* area) {
    k.mask = __activemask();
    k.lane = threadIdx.x & 31;
    k.below = (1u << k.lane) - 1u;
    k.nact = __popc(k.mask);
    k.rank = __popc(k.mask & k.below);
    k.leader = __ffs((int)k.mask) - 1;
    k.cbuf = area;
    k.rows = reinterpret_cast<unsigned long long*>(area + kKcMaxThr);
    k.claim = reinterpret_cast<int*>(k.rows + kKcMaxThr);
    // the group's earlier writes (a set a lane has just materialised) become visible to all of it
    __syncwarp(k.mask);
    int got = 0;
    if (k.lane == k.leader) got = atomicCAS(k.claim, 0, 1) == 0 ? 1 : 0;
    return __shfl_sync(k.mask, got, k.leader) != 0;
}
__device__ __forceinline__ void kc_coop_end(const KcCoop& k) {
    __syncwarp(k.mask);
    if (k.lane == k.leader) atomicExch(k.claim, 0);
}

// C = S n L by the lanes of the group (S the shorter sorted list, split over the
// lanes; L searched), kept in order in the area (up to kKcMaxThr members).
template <bool SSET, bool LSET>
__device__ __forceinline__ int kc_coop_collect(const KcCoop& k, const int* S, int ns, const int* L, int nl) {
    int cn = 0;
    for (int b = 0; b < ns; b += k.nact) {
        const int j = b + k.rank;
        int x = 0;
        bool in = false;
        if (j < ns) {
            x = kc_ld<SSET>(S + j);
            in = kc_contains<LSET>(L, nl, x);
        }
        const unsigned bal = __ballot_sync(k.mask, in);
        if (in) {
            const int p = cn + __popc(bal & k.below);
            if (p < kKcMaxThr) k.cbuf[p] = x;   // C in ascending order (S is sorted, lanes in rank order)
        }
        cn += __popc(bal);
    }
    return cn;
}

// One item, by all lanes of the group: C = A n B (sorted lists of the owner's
// graph, B an out-list; A in the scratch arena when ASET, read through L2),
// kept in order in the area; for need >= 2 and |C| <= thr also the rows of the
// subgraph C induces, and the owner's count from them.  Returns |C|; *add gets
// the owner's count (need == 1: |C|; 0 when C is larger than thr).
template <bool ASET>
__device__ __forceinline__ int kc_coop_item(const KcCoop& k, int owner, const int* A, int na, const int* B, int nb,
                                            const long long* goff, const int* gadj, int need, int thr,
                                            unsigned long long* add) {
    const int cn = (na <= nb) ? kc_coop_collect<ASET, false>(k, A, na, B, nb)
                              : kc_coop_collect<false, ASET>(k, B, nb, A, na);
    __syncwarp(k.mask);
    *add = 0;
    if (need == 1) {
        *add = (k.lane == owner) ? (unsigned long long)cn : 0ull;
    } else if (cn >= need && cn <= thr) {
        for (int a2 = 0; a2 < cn; ++a2) {
            const int w = k.cbuf[a2];
            const long long ow = __ldg(goff + w);
            const int nw = (int)(__ldg(goff + w + 1) - ow);
            unsigned long long bits = 0;
            for (int b = k.rank; b < nw; b += k.nact) {
                const int idx = kc_index_of(k.cbuf, cn, __ldg(gadj + ow + b));
                if (idx >= 0) bits |= 1ull << idx;
            }
            const unsigned r0 = __reduce_or_sync(k.mask, (unsigned)bits);
            const unsigned r1 = __reduce_or_sync(k.mask, (unsigned)(bits >> 32));
            if (k.rank == 0) k.rows[a2] = ((unsigned long long)r1 << 32) | r0;
        }
        __syncwarp(k.mask);
        if (k.lane == owner) *add = kc_count_rows(k.rows, cn, need);
    }
    __syncwarp(k.mask);   // the area is rewritten by the next item
    return cn;
}

// Warp-cooperative passes (orientation, where C's rows are built: at least two
// vertices still to choose): the lanes of a warp that reach the same task step
// take every such lane's items (DAG edges of a range step, branches of a set
// step) one after another, all together, so that lanes with short and long
// adjacency lists no longer wait for each other.  Per item the
// shorter list's elements are split over the lanes and looked up by binary
// search in the longer one; the rows of a small C are built the same way, one
// member's out-list per round.  Items whose C exceeds split_threshold go back
// to their owner lane (di / dc, at most hi - lo of them), which spawns them.
// Lanes of one warp may run tasks of different roots (batched or served
// graphs), so an item's graph, k and threshold are broadcast from its owner.
// Per-warp area: C (kKcMaxThr ints), its rows (kKcMaxThr words), a claim word.
constexpr int kKcCoopSmem = kKcMaxThr * 4 + kKcMaxThr * 8 + 16;

__device__ __forceinline__ const int* kc_bcast_ptr(unsigned mask, const void* p, int owner) {
    return reinterpret_cast<const int*>(__shfl_sync(mask, reinterpret_cast<unsigned long long>(p), owner));
}

// Range step: the DAG edges [lo, hi) of this lane.  Returns false, having done
// nothing, when the warp's area is in use.
static __device__ __noinline__ bool kc_coop_edges(const gtap_kclique_args& e, int* area, uint32_t lo, uint32_t hi,
                                                  int need, int thr, uint32_t* di, int* dc, int* dn,
                                                  unsigned long long* local) {
    KcCoop k;
    if (!kc_coop_begin(k, area)) return false;
    unsigned long long mine = 0;
    int nd = 0;
    for (unsigned m = k.mask; m != 0u; m &= m - 1u) {
        const int owner = __ffs((int)m) - 1;
        const uint32_t olo = __shfl_sync(k.mask, lo, owner), ohi = __shfl_sync(k.mask, hi, owner);
        const long long* goff = reinterpret_cast<const long long*>(kc_bcast_ptr(k.mask, e.off, owner));
        const int* gadj = kc_bcast_ptr(k.mask, e.adj, owner);
        const int* gsrc = kc_bcast_ptr(k.mask, e.src, owner);
        const int oneed = __shfl_sync(k.mask, need, owner), othr = __shfl_sync(k.mask, thr, owner);
        for (uint32_t ei = olo; ei < ohi; ++ei) {
            const int u = __ldg(gsrc + ei), v = __ldg(gadj + ei);
            const long long ou = __ldg(goff + u), ov = __ldg(goff + v);
            const int nu = (int)(__ldg(goff + u + 1) - ou), nv = (int)(__ldg(goff + v + 1) - ov);
            unsigned long long add;
            const int cn = kc_coop_item<false>(k, owner, gadj + ou, nu, gadj + ov, nv, goff, gadj, oneed, othr, &add);
            mine += add;
            if (k.lane == owner && oneed >= 2 && cn >= oneed && cn > othr) {
                di[nd] = ei;
                dc[nd] = cn;
                ++nd;
            }
        }
    }
    kc_coop_end(k);
    *dn = nd;
    *local = mine;
    return true;
}

// Set step: the branches [lo, hi) of this lane's set (len members, in the
// scratch arena).  Returns false, having done nothing, when the area is in use.
static __device__ __noinline__ bool kc_coop_branches(const gtap_kclique_args& e, int* area, const int* set, uint32_t len,
                                                     uint32_t lo, uint32_t hi, int need, int thr, uint32_t* di, int* dc,
                                                     int* dn, unsigned long long* local) {
    KcCoop k;
    if (!kc_coop_begin(k, area)) return false;
    unsigned long long mine = 0;
    int nd = 0;
    for (unsigned m = k.mask; m != 0u; m &= m - 1u) {
        const int owner = __ffs((int)m) - 1;
        const uint32_t olo = __shfl_sync(k.mask, lo, owner), ohi = __shfl_sync(k.mask, hi, owner);
        const uint32_t olen = __shfl_sync(k.mask, len, owner);
        const int* oset = kc_bcast_ptr(k.mask, set, owner);
        const long long* goff = reinterpret_cast<const long long*>(kc_bcast_ptr(k.mask, e.off, owner));
        const int* gadj = kc_bcast_ptr(k.mask, e.adj, owner);
        const int oneed = __shfl_sync(k.mask, need, owner), othr = __shfl_sync(k.mask, thr, owner);
        for (uint32_t i = olo; i < ohi; ++i) {
            const int w = __ldcg(oset + i);
            const long long ow = __ldg(goff + w);
            const int nw = (int)(__ldg(goff + w + 1) - ow);
            unsigned long long add;
            const int cn = kc_coop_item<true>(k, owner, oset, (int)olen, gadj + ow, nw, goff, gadj, oneed, othr, &add);
            mine += add;
            if (k.lane == owner && oneed >= 2 && cn >= oneed && cn > othr) {
                di[nd] = i;
                dc[nd] = cn;
                ++nd;
            }
        }
    }
    kc_coop_end(k);
    *dn = nd;
    *local = mine;
    return true;
}

static __device__ void kclique_range_step(TaskCtx& c) {
    const KcRangeSpawn a = c.load<KcRangeSpawn>();
    const gtap_kclique_args& e = kc_env(c.P, a.root);
    if (c.pc() != 0) { c.ret(a.acc + a.local); return; }
    const uint32_t n = a.hi - a.lo;
    if (n > (uint32_t)kKcFan) {
        const uint32_t per = (n + kKcFan - 1) / kKcFan;
        for (uint32_t s = a.lo; s < a.hi; s += per)
            c.spawn(T_KCLIQUE_ROOT, kKcRangeSlotAcc, kc_queue(e, 0), KcRangeSpawn{a.root, s, min(a.hi, s + per), 0u, 0ull, 0ull},
                    kFlagAccumulate);
        c.join(1, kc_queue(e, 0));
        return;
    }
    const int thr = e.split_threshold;
    const int need = e.k - 2;
    const bool pivot = e.algorithm == GTAP_KCLIQUE_PIVOT;
    unsigned long long local = 0;
    uint32_t dei[kKcFan];
    int dcn[kKcFan];
    int dn = 0;
    if (!pivot && need >= 2 &&
        kc_coop_edges(e, reinterpret_cast<int*>(c.ws.prog), a.lo, a.hi, need, thr, dei, dcn, &dn, &local)) {
        // orientation, warp-cooperative pass done; the sets too large to count there become set tasks
        for (int q = 0; q < dn; ++q) {
            const uint32_t ei = dei[q];
            const int u = __ldg(e.src + ei), v = __ldg(e.adj + ei);
            const long long ou = kc_off(e, u);
            const int nu = (int)(kc_off(e, u + 1) - ou);
            c.spawn(T_KCLIQUE_SET, kKcRangeSlotAcc, kc_queue(e, 1),
                    KcSetSpawn{a.root, (uint32_t)need, (unsigned long long)(e.adj + ou), (uint32_t)nu, (uint32_t)v,
                               (uint32_t)dcn[q], kKcLazy, 0ull, 0ull},
                    kFlagAccumulate);
        }
        if (c.nspawned == 0) { c.ret(local); return; }
        st_cg64(c.frame + kKcRangeLocal, local);
        c.join(1, kc_queue(e, 0));
        return;
    }
    int C[kKcMaxThr];
    for (uint32_t ei = a.lo; ei < a.hi; ++ei) {
        const int u = __ldg(e.src + ei), v = __ldg(e.adj + ei);
        const long long ou = kc_off(e, u), ov = kc_off(e, v);
        const int nu = (int)(kc_off(e, u + 1) - ou), nv = (int)(kc_off(e, v + 1) - ov);
        const int cn = kc_intersect(e.adj + ou, nu, AdjLoad{}, e.adj + ov, nv, AdjLoad{}, C, pivot ? kKcMaxThr : thr);
        if (need == 1) { local += (unsigned)cn; continue; }
        if (cn < need) continue;
        if (cn <= thr) {
            local += pivot ? kp_count_small(C, cn, need, e.off, e.adj) : kc_count_small(C, cn, need, e.off, e.adj);
            continue;
        }
        if (pivot && cn <= kKcMaxThr) {
            if (!kp_spawn_split(c, e, a.root, C, cn, need, 1, kKcRangeSlotAcc)) return;
            continue;
        }
        if (pivot) {
            // more than 64 members: a pivot node over multi-word bitsets, materialised when it runs
            c.spawn(T_KCLIQUE_PIVB, kKcRangeSlotAcc, kc_queue(e, 1),
                    KpbSpawn{a.root, (uint32_t)need | (kKpbLazy << 24), (unsigned long long)(e.adj + ou),
                             (unsigned long long)(uint32_t)v | ((unsigned long long)(uint32_t)nu << 32),
                             kpb_range((uint32_t)cn, (uint32_t)cn, 0, 1), 0ull, 0ull},
                    kFlagAccumulate);
            continue;
        }
        // the child materialises N+(u) n N+(v) when it runs and adds its count
        // into this range task's accumulator
        c.spawn(T_KCLIQUE_SET, kKcRangeSlotAcc, kc_queue(e, 1),
                KcSetSpawn{a.root, (uint32_t)need, (unsigned long long)(e.adj + ou), (uint32_t)nu, (uint32_t)v, (uint32_t)cn,
                           kKcLazy, 0ull, 0ull},
                kFlagAccumulate);
    }
    if (c.nspawned == 0) { c.ret(local); return; }
    st_cg64(c.frame + kKcRangeLocal, local);
    c.join(1, kc_queue(e, 0));
}

// COOP: the warp-cooperative branch pass is compiled in (the dispatcher picks it
// for orientation steps that build rows); without it the per-lane step keeps
// the registers it had.
template <bool COOP>
static __device__ void kclique_set_step(TaskCtx& c) {
    const KcSetSpawn a = c.load<KcSetSpawn>();
    const gtap_kclique_args& e = kc_env(c.P, a.root);
    if (c.pc() != 0) {
        // an owner frees its set once every task that reads it is done
        if (a.own == 1u) scratch_free(c.P, reinterpret_cast<const int*>(a.set), c.type(), c.worker);
        c.ret(a.acc + a.local);
        return;
    }
    const int* set = reinterpret_cast<const int*>(a.set);
    uint32_t len = a.len, lo = a.lo, hi = a.hi, own = a.own;
    if (own == kKcLazy) {
        // materialise S = P n N+(w) (|S| = hi > thr, known from the spawn)
        const int w = (int)a.lo;
        const long long ow = kc_off(e, w);
        const int nw = (int)(kc_off(e, w + 1) - ow);
        bool pooled;
        int* S = kc_scratch_alloc(c, (int)a.hi, &pooled);
        if (!S) return;
        kc_intersect(set, (int)a.len, SetLoad{}, e.adj + ow, nw, AdjLoad{}, S, (int)a.hi);
        set = S;
        len = a.hi;
        lo = 0;
        own = pooled ? 1u : 0u;
        // what the resume needs: the set to free
        st_cg64(c.frame + kKcSetPtr, (unsigned long long)S);
        st_cg64(c.frame + kKcSetLenLo, (unsigned long long)len);
        st_cg64(c.frame + kKcSetHiOwn, (unsigned long long)hi | ((unsigned long long)own << 32));
    }
    const int depth = e.k - 2 - (int)a.j + 1;
    const uint32_t n = hi - lo;
    if (n > (uint32_t)kKcFan) {
        const uint32_t per = (n + kKcFan - 1) / kKcFan;
        for (uint32_t s = lo; s < hi; s += per)
            c.spawn(T_KCLIQUE_SET, kKcSetSlotAcc, kc_queue(e, depth),
                    KcSetSpawn{a.root, a.j, (unsigned long long)set, len, s, min(hi, s + per), 0u, 0ull, 0ull},
                    kFlagAccumulate);
        c.join(1, kc_queue(e, depth));
        return;
    }
    const int thr = e.split_threshold;
    const int need = (int)a.j - 1;
    const bool pivot = e.algorithm == GTAP_KCLIQUE_PIVOT;
    unsigned long long local = 0;
    uint32_t di[kKcFan];
    int dc[kKcFan];
    int dn = 0;
    // cooperative only where C's rows are built (need >= 2): a count alone (need == 1) is one
    // latency-bound search per branch, better overlapped across the lanes' own branches
    if (COOP && !pivot && need >= 2 &&
        kc_coop_branches(e, reinterpret_cast<int*>(c.ws.prog), set, len, lo, hi, need, thr, di, dc, &dn, &local)) {
        // orientation, warp-cooperative pass done; this lane materialises and spawns its larger sets
        for (int q = 0; q < dn; ++q) {
            const int w = __ldcg(set + di[q]);
            const long long ow = kc_off(e, w);
            const int nw = (int)(kc_off(e, w + 1) - ow);
            bool pooled;
            int* S = kc_scratch_alloc(c, dc[q], &pooled);
            if (!S) return;
            kc_intersect(set, (int)len, SetLoad{}, e.adj + ow, nw, AdjLoad{}, S, dc[q]);
            c.spawn(T_KCLIQUE_SET, kKcSetSlotAcc, kc_queue(e, depth + 1),
                    KcSetSpawn{a.root, (uint32_t)need, (unsigned long long)S, (uint32_t)dc[q], 0u, (uint32_t)dc[q],
                               pooled ? 1u : 0u, 0ull, 0ull},
                    kFlagAccumulate);
        }
        hi = lo;   // the per-lane loop below has nothing left to do
    }
    int C[kKcMaxThr];
    for (uint32_t i = lo; i < hi; ++i) {
        const int w = __ldcg(set + i);
        const long long ow = kc_off(e, w);
        const int nw = (int)(kc_off(e, w + 1) - ow);
        const int cn = kc_intersect(set, (int)len, SetLoad{}, e.adj + ow, nw, AdjLoad{}, C, pivot ? kKcMaxThr : thr);
        if (need == 1) { local += (unsigned)cn; continue; }
        if (cn < need) continue;
        if (cn <= thr) {
            local += pivot ? kp_count_small(C, cn, need, e.off, e.adj) : kc_count_small(C, cn, need, e.off, e.adj);
            continue;
        }
        if (pivot && cn <= kKcMaxThr) {
            if (!kp_spawn_split(c, e, a.root, C, cn, need, depth + 1, kKcSetSlotAcc)) return;
            continue;
        }
        // deeper sets are materialised here, by the spawning lane (see the header)
        bool pooled;
        int* S = kc_scratch_alloc(c, cn, &pooled);
        if (!S) return;
        kc_intersect(set, (int)len, SetLoad{}, e.adj + ow, nw, AdjLoad{}, S, cn);
        c.spawn(T_KCLIQUE_SET, kKcSetSlotAcc, kc_queue(e, depth + 1),
                KcSetSpawn{a.root, (uint32_t)need, (unsigned long long)S, (uint32_t)cn, 0u, (uint32_t)cn, pooled ? 1u : 0u,
                           0ull, 0ull},
                kFlagAccumulate);
    }
    if (c.nspawned == 0) {
        if (own == 1u) scratch_free(c.P, set, c.type(), c.worker);
        c.ret(local);
        return;
    }
    st_cg64(c.frame + kKcSetLocal, local);
    c.join(1, kc_queue(e, depth));
}

// A set step whose branches still need at least two more vertices (j >= 3) runs
// the cooperative pass (orientation only); the rest take the lean per-lane step.
__device__ __forceinline__ void kclique_set_dispatch(TaskCtx& c) {
    const unsigned long long w2 = c.word<2>();   // record bytes 16..23: root, j
    const uint32_t j = (uint32_t)(w2 >> 32);
    if (c.pc() == 0 && j >= 3 && kc_env(c.P, (uint32_t)w2).algorithm != GTAP_KCLIQUE_PIVOT) kclique_set_step<true>(c);
    else kclique_set_step<false>(c);
}

}  // namespace gtap

namespace gtap {

// ---------------------------------------------------------------------------
// Thread-mode Cilksort (Sec. 6.3: sort halves in parallel and merge with a
// forked parallel merge; Sec. 6.3.2 routes recursive, serial-sort and
// serial-merge tasks to three DAQ queues).  One lane is one task, so a leaf
// sorts or merges its keys alone (these lanes touch unrelated data: the
// accesses of a warp are not coalesced, the structural cost the paper names).
// Buffers: 0 = dst, 1 = tmp; sort leaves read src.
// Records:  TSORT  [16] root, into  [24] lo, hi (u32)
//           TMERGE [16] root, from  [24] a0, a1, b0, b1  [40] out
struct CsSortSpawn { uint32_t root, into, lo, hi; };
struct CsMergeSpawn { uint32_t root, from, a0, a1, b0, b1, out, pad; };
constexpr uint32_t kCsSlot = 7;       // void results: accumulate 0, nothing written
constexpr int kCsMaxSortCut = 256;

__device__ __forceinline__ gtap_cilksort_args cs_env(const KParams& P, uint32_t root) {
    return P.serving ? ld_obj<gtap_cilksort_args>(P.root_desc[root].env)
                     : ld_obj_ro<gtap_cilksort_args>(P.root_desc[root].env);
}
__device__ __forceinline__ uint32_t* cs_buf(const gtap_cilksort_args& e, uint32_t b) { return b ? e.tmp : e.dst; }
__device__ __forceinline__ int cs_queue(const gtap_cilksort_args& e, int kind) { return e.route ? kind : 0; }

__device__ __forceinline__ void cs_merge_spawn(TaskCtx& c, const gtap_cilksort_args& e, uint32_t root, uint32_t from,
                                               uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1, uint32_t out) {
    const bool leaf = (a1 - a0) + (b1 - b0) <= e.merge_cutoff;
    c.spawn(T_TMERGE, kCsSlot, cs_queue(e, leaf ? 2 : 0), CsMergeSpawn{root, from, a0, a1, b0, b1, out, 0u},
            kFlagAccumulate);
}

__device__ __forceinline__ void cilksort_sort_step(TaskCtx& c) {
    const CsSortSpawn a = c.load<CsSortSpawn>();
    const gtap_cilksort_args e = cs_env(c.P, a.root);
    const uint32_t n = a.hi - a.lo, mid = a.lo + n / 2;
    if (c.pc() == 0) {
        if (n <= e.sort_cutoff) {
            // serial leaf: insertion sort of the range in the lane's local memory
            uint32_t k[kCsMaxSortCut];
            for (uint32_t i = 0; i < n; ++i) {
                const uint32_t x = __ldcg(e.src + a.lo + i);
                uint32_t j = i;
                while (j > 0 && k[j - 1] > x) { k[j] = k[j - 1]; --j; }
                k[j] = x;
            }
            uint32_t* out = cs_buf(e, a.into) + a.lo;
            for (uint32_t i = 0; i < n; ++i) __stcg(out + i, k[i]);
            c.ret(0ull);
            return;
        }
        const uint32_t other = 1u - a.into;
        const uint32_t h0 = mid - a.lo, h1 = a.hi - mid;
        c.spawn(T_TSORT, kCsSlot, cs_queue(e, h0 <= e.sort_cutoff ? 1 : 0), CsSortSpawn{a.root, other, a.lo, mid}, kFlagAccumulate);
        c.spawn(T_TSORT, kCsSlot, cs_queue(e, h1 <= e.sort_cutoff ? 1 : 0), CsSortSpawn{a.root, other, mid, a.hi}, kFlagAccumulate);
        c.join(1, 0);
    } else if (c.pc() == 1) {
        // the halves are sorted in the other buffer: merge them back into this task's buffer
        cs_merge_spawn(c, e, a.root, 1u - a.into, a.lo, mid, mid, a.hi, a.lo);
        c.join(2, 0);
    } else {
        c.ret(0ull);
    }
}

__device__ __forceinline__ void cilksort_merge_step(TaskCtx& c) {
    const CsMergeSpawn a = c.load<CsMergeSpawn>();
    if (c.pc() != 0) { c.ret(0ull); return; }
    const gtap_cilksort_args e = cs_env(c.P, a.root);
    const uint32_t* X = cs_buf(e, a.from);
    uint32_t* Y = cs_buf(e, 1u - a.from);
    uint32_t a0 = a.a0, a1 = a.a1, b0 = a.b0, b1 = a.b1;
    if ((a1 - a0) + (b1 - b0) <= e.merge_cutoff) {
        // serial leaf: two-finger merge
        uint32_t i = a0, j = b0, k = a.out;
        uint32_t x = i < a1 ? __ldcg(X + i) : 0u, y = j < b1 ? __ldcg(X + j) : 0u;
        while (i < a1 && j < b1) {
            if (y < x) { __stcg(Y + k++, y); if (++j < b1) y = __ldcg(X + j); }
            else { __stcg(Y + k++, x); if (++i < a1) x = __ldcg(X + i); }
        }
        for (; i < a1; ++i) __stcg(Y + k++, __ldcg(X + i));
        for (; j < b1; ++j) __stcg(Y + k++, __ldcg(X + j));
        c.ret(0ull);
        return;
    }
    if (a1 - a0 < b1 - b0) { uint32_t t = a0; a0 = b0; b0 = t; t = a1; a1 = b1; b1 = t; }
    const uint32_t ma = a0 + (a1 - a0) / 2;
    const uint32_t x = __ldcg(X + ma);
    uint32_t lo = b0, hi = b1;   // first position of B whose key is not less than x
    while (lo < hi) { const uint32_t m = lo + (hi - lo) / 2; if (__ldcg(X + m) < x) lo = m + 1; else hi = m; }
    const uint32_t at = a.out + (ma - a0) + (lo - b0);
    __stcg(Y + at, x);
    cs_merge_spawn(c, e, a.root, a.from, a0, ma, b0, lo, a.out);
    cs_merge_spawn(c, e, a.root, a.from, ma + 1, a1, lo, b1, at + 1);
    c.join(1, 0);
}

}  // namespace gtap
