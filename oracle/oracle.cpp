// CPU oracle for the GTaP fork-join workloads.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, sequential
// statement of what each task program computes.  It is used by the tests, by
// the package's smoke check and by the bench's CPU-baseline leg, never by the
// library's compute path, and it shares no code, header or constant table
// with the CUDA sources.
//
// Every integer program is the *serial elision* of its task program: each
// fork ("task") becomes an ordinary call and each join ("taskwait") a no-op.
// The paper states that the queue clause does not change a program's meaning
// (Sec. 4.2, DAQ) and fork-join over these programs is deterministic, so the
// GPU runtime must reach exactly these results.  Each routine also counts the
// task invocations the GPU program creates, so the task counts can be
// compared too.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -shared -fPIC (no fused
// multiply-add, so floating-point programs round at every operation).
//
// Parity status per routine (see tests/test_oracle_pins.py):
//   fib, nqueens, uts, sort, cilksort, integrate, kclique (orientation and pivoting), bintree: pinned.
//   fmm: pinned against the direct O(N^2) sum (exact regime and convergence).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the state advances by the
// golden-ratio increment and the output is a 3-step xor-shift-multiply
// finaliser.  splitmix64(x) below is "advance once from state x, then mix",
// i.e. the first output of a stream seeded x.
uint64_t sm64_finalize(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
uint64_t splitmix64(uint64_t x) { return sm64_finalize(x + 0x9E3779B97F4A7C15ULL); }

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// SplitMix64 stream output k of seed s (for the golden-vector pin).
uint64_t orc_splitmix64_next(uint64_t state_before) { return splitmix64(state_before); }

// ---------------------------------------------------------------------------
// Fibonacci, no cutoff (Sec. 6.3, "Fibonacci": a task at every recursive call).
// fib(n) = n for n < 2, else fib(n-1) + fib(n-2), summed in int64.
static int64_t fib_rec(int n, uint64_t* tasks) {
    ++*tasks;
    if (n < 2) return n;
    int64_t l = fib_rec(n - 1, tasks);  // task
    int64_t r = fib_rec(n - 2, tasks);  // task
    return l + r;                        // after taskwait
}
int64_t orc_fib(int n, uint64_t* tasks) {
    uint64_t t = 0;
    int64_t v = fib_rec(n, &t);
    if (tasks) *tasks = t;
    return v;
}

// Fibonacci with a sequential cutoff (Sec. 6.3.2, the DAQ experiment): a call
// with n >= cutoff (and n >= 2) is a task that forks its two calls; a call
// with n below the cutoff is a leaf task that computes fib(n) by the plain
// serial recursion.  The value is unchanged; the task count is the number of
// calls with n >= cutoff plus the leaf calls they make.
static int64_t fib_serial(int n) { return n < 2 ? n : fib_serial(n - 1) + fib_serial(n - 2); }
static int64_t fib_cut(int n, int cutoff, uint64_t* tasks) {
    ++*tasks;
    if (n < 2 || n < cutoff) return fib_serial(n);
    return fib_cut(n - 1, cutoff, tasks) + fib_cut(n - 2, cutoff, tasks);
}
int64_t orc_fib_cutoff(int n, int cutoff, uint64_t* tasks) {
    uint64_t t = 0;
    int64_t v = fib_cut(n, cutoff, &t);
    if (tasks) *tasks = t;
    return v;
}

// ---------------------------------------------------------------------------
// N-Queens by bitmask backtracking (Sec. 6.3, "N-Queens"), one task per
// placed row: the root is the empty board at row 0, and a task at row r
// spawns one child for every column where a queen in row r is not attacked.
// A task at row n is a solution.  Nodes counts every task (root included).
static void nq_bits(int n, int row, uint32_t cols, uint32_t diag_l, uint32_t diag_r,
                    uint64_t* sols, uint64_t* nodes) {
    ++*nodes;
    if (row == n) { ++*sols; return; }
    const uint32_t full = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
    uint32_t avail = ~(cols | diag_l | diag_r) & full;
    while (avail) {
        uint32_t bit = avail & (0u - avail);
        avail ^= bit;
        nq_bits(n, row + 1, cols | bit, (diag_l | bit) << 1, (diag_r | bit) >> 1, sols, nodes);
    }
}
uint64_t orc_nqueens_bitmask(int n, uint64_t* nodes) {
    uint64_t s = 0, t = 0;
    nq_bits(n, 0, 0, 0, 0, &s, &t);
    if (nodes) *nodes = t;
    return s;
}

// N-Queens with a cutoff depth (Sec. 6.3.1 uses depth 7): a board with fewer
// than `depth` rows placed is a task that forks one child per legal placement
// in the next row; a board with `depth` rows placed (or a complete board) is a
// leaf task that finishes the search serially.  Tasks = boards with at most
// `depth` rows placed.
static uint64_t nq_serial(int n, int row, uint32_t cols, uint32_t dl, uint32_t dr) {
    if (row == n) return 1;
    uint64_t s = 0;
    const uint32_t full = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
    for (uint32_t avail = ~(cols | dl | dr) & full; avail; avail &= avail - 1) {
        uint32_t bit = avail & (0u - avail);
        s += nq_serial(n, row + 1, cols | bit, (dl | bit) << 1, (dr | bit) >> 1);
    }
    return s;
}
static uint64_t nq_cut(int n, int depth, int row, uint32_t cols, uint32_t dl, uint32_t dr, uint64_t* tasks) {
    ++*tasks;
    if (row == n || row >= depth) return nq_serial(n, row, cols, dl, dr);
    uint64_t s = 0;
    const uint32_t full = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
    for (uint32_t avail = ~(cols | dl | dr) & full; avail; avail &= avail - 1) {
        uint32_t bit = avail & (0u - avail);
        s += nq_cut(n, depth, row + 1, cols | bit, (dl | bit) << 1, (dr | bit) >> 1, tasks);
    }
    return s;
}
uint64_t orc_nqueens_cutoff(int n, int depth, uint64_t* tasks) {
    uint64_t t = 0;
    uint64_t s = nq_cut(n, depth, 0, 0, 0, 0, &t);
    if (tasks) *tasks = t;
    return s;
}

// Independent second algorithm: queens stored as a column array, attacks
// checked pairwise, no bit tricks.  Same tree, so the same node count.
static void nq_array(int n, int row, int* q, uint64_t* sols, uint64_t* nodes) {
    ++*nodes;
    if (row == n) { ++*sols; return; }
    for (int c = 0; c < n; ++c) {
        bool ok = true;
        for (int r = 0; r < row && ok; ++r) {
            int dc = q[r] - c;
            if (dc < 0) dc = -dc;
            if (q[r] == c || dc == row - r) ok = false;
        }
        if (ok) { q[row] = c; nq_array(n, row + 1, q, sols, nodes); }
    }
}
uint64_t orc_nqueens_array(int n, uint64_t* nodes) {
    std::vector<int> q(n > 0 ? n : 1);
    uint64_t s = 0, t = 0;
    nq_array(n, 0, q.data(), &s, &t);
    if (nodes) *nodes = t;
    return s;
}

// Brute force: every permutation of columns (one queen per row and column),
// keeping those with no two queens on a diagonal.
uint64_t orc_nqueens_permutations(int n) {
    std::vector<int> p(n);
    for (int i = 0; i < n; ++i) p[i] = i;
    uint64_t count = 0;
    if (n == 0) return 1;
    do {
        bool ok = true;
        for (int i = 0; i < n && ok; ++i)
            for (int j = i + 1; j < n && ok; ++j)
                if (std::abs(p[i] - p[j]) == j - i) ok = false;
        if (ok) ++count;
    } while (std::next_permutation(p.begin(), p.end()));
    return count;
}

// ---------------------------------------------------------------------------
// Unbalanced hashed tree (the UTS-like workload of the integer benchmark
// set).  Node ids: root = splitmix64(seed); child i (0-based) of p =
// splitmix64(p ^ (0x9E3779B97F4A7C15 * (i + 1))).  The root has
// root_children children; any other node v has m children iff
// splitmix64(v ^ 0xD1B54A32D192ED03) < threshold, else none.
static uint64_t uts_child(uint64_t parent, uint32_t i) {
    return splitmix64(parent ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(i + 1)));
}
static uint32_t uts_arity(uint64_t v, uint32_t m, uint64_t threshold) {
    return splitmix64(v ^ 0xD1B54A32D192ED03ULL) < threshold ? m : 0u;
}
struct UtsTotals { uint64_t nodes, leaves, max_depth; };
static void uts_rec(uint64_t v, uint32_t arity, uint32_t m, uint64_t thr, uint64_t depth, UtsTotals* t) {
    ++t->nodes;
    if (depth > t->max_depth) t->max_depth = depth;
    if (arity == 0) { ++t->leaves; return; }
    for (uint32_t i = 0; i < arity; ++i) {
        uint64_t c = uts_child(v, i);
        uts_rec(c, uts_arity(c, m, thr), m, thr, depth + 1, t);
    }
}
void orc_uts_recursive(uint64_t seed, uint32_t root_children, uint32_t m, uint64_t threshold,
                       uint64_t* nodes, uint64_t* leaves, uint64_t* max_depth) {
    UtsTotals t{0, 0, 0};
    uts_rec(splitmix64(seed), root_children, m, threshold, 0, &t);
    *nodes = t.nodes; *leaves = t.leaves;
    if (max_depth) *max_depth = t.max_depth;
}
// Independent traversal: breadth-first with an explicit FIFO, no recursion.
void orc_uts_bfs(uint64_t seed, uint32_t root_children, uint32_t m, uint64_t threshold,
                 uint64_t* nodes, uint64_t* leaves) {
    std::vector<uint64_t> frontier{splitmix64(seed)}, next;
    uint64_t n = 0, l = 0;
    bool root_level = true;
    while (!frontier.empty()) {
        next.clear();
        for (uint64_t v : frontier) {
            ++n;
            uint32_t a = root_level ? root_children : uts_arity(v, m, threshold);
            if (a == 0) ++l;
            for (uint32_t i = 0; i < a; ++i) next.push_back(uts_child(v, i));
        }
        root_level = false;
        frontier.swap(next);
    }
    *nodes = n; *leaves = l;
}

// ---------------------------------------------------------------------------
// Mergesort (Cilksort, Sec. 6.3): the result of any correct sort is the
// ascending order of the keys; the library sort is the oracle.
void orc_sort_u32(const uint32_t* in, uint32_t* out, uint64_t n) {
    std::memcpy(out, in, n * sizeof(uint32_t));
    std::sort(out, out + n);
}

// Thread-mode Cilksort (Sec. 6.3, "Cilksort parallelizes merging"; Sec.
// 6.3.2 runs it with three DAQ queues: recursive, serial-sort and
// serial-merge tasks).  sort(range, into): a range of at most sort_cutoff keys
// is a leaf task that sorts it serially into buffer `into`; a larger range
// forks its two halves into the other buffer and then merges them into `into`.
// merge(A, B -> out): at most merge_cutoff outputs is a leaf task that merges
// serially; otherwise the longer run's middle element x is written straight
// to its final place (after the keys of A before it and the keys of B less
// than x), and the two sub-merges on either side of it are forked, so each
// has fewer outputs than its parent.  The sorted output is whatever a correct
// sort gives; the task count is that of this recursion.
struct CilkState { std::vector<uint32_t> buf[2]; const uint32_t* src; uint64_t sort_cut, merge_cut, tasks; };

static void cilk_merge(CilkState& st, int from, uint64_t a0, uint64_t a1, uint64_t b0, uint64_t b1, uint64_t out) {
    ++st.tasks;
    const std::vector<uint32_t>& X = st.buf[from];
    std::vector<uint32_t>& Y = st.buf[1 - from];
    uint64_t na = a1 - a0, nb = b1 - b0;
    if (na + nb <= st.merge_cut) {
        // plain two-finger merge
        uint64_t i = a0, j = b0, k = out;
        while (i < a1 && j < b1) Y[k++] = (X[j] < X[i]) ? X[j++] : X[i++];
        while (i < a1) Y[k++] = X[i++];
        while (j < b1) Y[k++] = X[j++];
        return;
    }
    if (na < nb) { std::swap(a0, b0); std::swap(a1, b1); std::swap(na, nb); }
    const uint64_t ma = a0 + na / 2;
    const uint32_t x = X[ma];
    // first position of the shorter run whose key is not less than x
    const uint64_t mb = (uint64_t)(std::lower_bound(X.begin() + b0, X.begin() + b1, x) - X.begin());
    const uint64_t at = out + (ma - a0) + (mb - b0);
    Y[at] = x;
    cilk_merge(st, from, a0, ma, b0, mb, out);
    cilk_merge(st, from, ma + 1, a1, mb, b1, at + 1);
}

static void cilk_sort(CilkState& st, uint64_t lo, uint64_t hi, int into) {
    ++st.tasks;
    if (hi - lo <= st.sort_cut) {
        std::vector<uint32_t> part(st.src + lo, st.src + hi);
        std::sort(part.begin(), part.end());
        std::copy(part.begin(), part.end(), st.buf[into].begin() + lo);
        return;
    }
    const uint64_t mid = lo + (hi - lo) / 2;
    cilk_sort(st, lo, mid, 1 - into);
    cilk_sort(st, mid, hi, 1 - into);
    cilk_merge(st, 1 - into, lo, mid, mid, hi, lo);
}

// Sorts in[0, n) into out; returns the number of tasks the recursion creates.
uint64_t orc_cilksort(const uint32_t* in, uint32_t* out, uint64_t n, uint64_t sort_cutoff, uint64_t merge_cutoff) {
    CilkState st;
    st.buf[0].assign(n, 0);
    st.buf[1].assign(n, 0);
    st.src = in;
    st.sort_cut = sort_cutoff < 1 ? 1 : sort_cutoff;
    st.merge_cut = merge_cutoff < 1 ? 1 : merge_cutoff;
    st.tasks = 0;
    if (n > 0) cilk_sort(st, 0, n, 0);
    std::copy(st.buf[0].begin(), st.buf[0].end(), out);
    return st.tasks;
}

// ---------------------------------------------------------------------------
// Adaptive trapezoid integration with Richardson extrapolation (Program 1).
// The integrand is fixed to the Runge function 1/(1 + 25 x^2), written with
// + - * / only so that every step is correctly rounded on any IEEE machine.
static double runge(double x) { return 1.0 / (1.0 + (25.0 * x) * x); }
static double trap(double a, double b) { return ((b - a) * (runge(a) + runge(b))) * 0.5; }

// Thread mode, Program 1(a): one trapezoid for the coarse estimate, two for
// the fine one; accept when they agree within eps, else fork on the halves.
static double integ_thread(double a, double b, double eps, uint64_t* tasks) {
    ++*tasks;
    double m = 0.5 * (a + b);
    double coarse = trap(a, b);
    double fine = trap(a, m) + trap(m, b);
    if (std::fabs(fine - coarse) < eps) return (4.0 * fine - coarse) / 3.0;
    double l = integ_thread(a, m, eps, tasks);
    double r = integ_thread(m, b, eps, tasks);
    return l + r;
}
double orc_integrate_thread(double a, double b, double eps, uint64_t* tasks) {
    uint64_t t = 0;
    double v = integ_thread(a, b, eps, &t);
    if (tasks) *tasks = t;
    return v;
}

// Block mode, Program 1(b): block_trap(a, b, n) splits [a, b] into n equal
// trapezoids evaluated by the block's threads.  The paper does not fix the
// summation order; the one used here (and by the GPU program) is: node
// x_i = a + h*i (x_n = b), thread t sums trapezoids t, t+B, t+2B, ... in
// order, then the B partial sums are combined by the halving tree
// s[t] += s[t + s] for s = B/2, B/4, ..., 1.
static double block_trap(double a, double b, int n, int B) {
    double h = (b - a) / (double)n;
    std::vector<double> part(B, 0.0);
    for (int t = 0; t < B; ++t) {
        double s = 0.0;
        for (int i = t; i < n; i += B) {
            double x0 = a + h * (double)i;
            double x1 = (i + 1 == n) ? b : a + h * (double)(i + 1);
            s += ((x1 - x0) * (runge(x0) + runge(x1))) * 0.5;
        }
        part[t] = s;
    }
    for (int stride = B / 2; stride >= 1; stride /= 2)
        for (int t = 0; t < stride; ++t) part[t] += part[t + stride];
    return part[0];
}
static double integ_block(double a, double b, double eps, int B, uint64_t* tasks) {
    ++*tasks;
    const int NTRAP = 256;
    double coarse = block_trap(a, b, NTRAP, B);
    double fine = block_trap(a, b, 2 * NTRAP, B);
    if (std::fabs(fine - coarse) < eps) return (4.0 * fine - coarse) / 3.0;
    double m = 0.5 * (a + b);
    double l = integ_block(a, m, eps, B, tasks);
    double r = integ_block(m, b, eps, B, tasks);
    return l + r;
}
double orc_integrate_block(double a, double b, double eps, int block_size, uint64_t* tasks) {
    uint64_t t = 0;
    double v = integ_block(a, b, eps, block_size, &t);
    if (tasks) *tasks = t;
    return v;
}

// ---------------------------------------------------------------------------
// k-clique counting by graph orientation (Sec. 6.4.2).  Orient every
// undirected edge from the lower to the higher vertex of a total order
// (order_mode 0: (degree, id) lexicographic; 1: id), giving a DAG in which
// every k-clique appears exactly once as a chain.  For each directed edge
// (u, v) take C = N+(u) intersect N+(v) and count the (k-2)-cliques inside
// C: count(S, 1) = |S|, count(S, j) = sum over w in S of count(S n N+(w), j-1).
struct Dag { std::vector<int64_t> off; std::vector<int32_t> adj; };

static Dag orient(int64_t n, const int32_t* edges, int64_t m, int order_mode) {
    std::vector<int64_t> deg(n, 0);
    for (int64_t e = 0; e < m; ++e) { ++deg[edges[2 * e]]; ++deg[edges[2 * e + 1]]; }
    auto before = [&](int32_t a, int32_t b) {
        if (order_mode == 0 && deg[a] != deg[b]) return deg[a] < deg[b];
        return a < b;
    };
    Dag g;
    g.off.assign(n + 1, 0);
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        ++g.off[(before(a, b) ? a : b) + 1];
    }
    for (int64_t v = 0; v < n; ++v) g.off[v + 1] += g.off[v];
    g.adj.assign(m, 0);
    std::vector<int64_t> fill(g.off.begin(), g.off.end() - 1);
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (before(a, b)) g.adj[fill[a]++] = b; else g.adj[fill[b]++] = a;
    }
    for (int64_t v = 0; v < n; ++v) std::sort(g.adj.begin() + g.off[v], g.adj.begin() + g.off[v + 1]);
    return g;
}

static std::vector<int32_t> intersect(const int32_t* a, int64_t na, const int32_t* b, int64_t nb) {
    std::vector<int32_t> out;
    std::set_intersection(a, a + na, b, b + nb, std::back_inserter(out));
    return out;
}

static uint64_t count_in(const Dag& g, const std::vector<int32_t>& S, int j) {
    if (j == 1) return S.size();
    uint64_t total = 0;
    for (int32_t w : S) {
        std::vector<int32_t> T = intersect(S.data(), (int64_t)S.size(), g.adj.data() + g.off[w],
                                           g.off[w + 1] - g.off[w]);
        if ((int)T.size() >= j - 1) total += count_in(g, T, j - 1);
    }
    return total;
}

// Total count; per_edge (optional, length m) receives the count of each
// directed edge in DAG order (vertex u ascending, then its sorted out-list).
uint64_t orc_kclique(int64_t n, const int32_t* edges, int64_t m, int k, int order_mode,
                     uint64_t* per_edge) {
    if (k == 1) return (uint64_t)n;
    if (k == 2) { if (per_edge) for (int64_t e = 0; e < m; ++e) per_edge[e] = 1; return (uint64_t)m; }
    Dag g = orient(n, edges, m, order_mode);
    uint64_t total = 0;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t p = g.off[u]; p < g.off[u + 1]; ++p) {
            int32_t v = g.adj[p];
            std::vector<int32_t> C = intersect(g.adj.data() + g.off[u], g.off[u + 1] - g.off[u],
                                               g.adj.data() + g.off[v], g.off[v + 1] - g.off[v]);
            uint64_t c = ((int)C.size() >= k - 2) ? count_in(g, C, k - 2) : 0;
            if (per_edge) per_edge[p] = c;
            total += c;
        }
    }
    return total;
}

// Sum of the per-edge counts over DAG edges [lo, hi) (same edge order as above),
// so a sample of a large graph can be checked without counting every edge.
uint64_t orc_kclique_edge_range(int64_t n, const int32_t* edges, int64_t m, int k, int order_mode, int64_t lo,
                                int64_t hi) {
    Dag g = orient(n, edges, m, order_mode);
    uint64_t total = 0;
    int64_t u = 0;
    for (int64_t p = lo; p < hi && p < m; ++p) {
        while (g.off[u + 1] <= p) ++u;
        int32_t v = g.adj[p];
        std::vector<int32_t> C = intersect(g.adj.data() + g.off[u], g.off[u + 1] - g.off[u],
                                           g.adj.data() + g.off[v], g.off[v + 1] - g.off[v]);
        if (k == 3) total += C.size();
        else if ((int)C.size() >= k - 2) total += count_in(g, C, k - 2);
    }
    return total;
}

// Sum of the per-edge counts over several DAG-edge ranges [ranges[2i],
// ranges[2i+1]) of a graph already oriented (off/adj as orc_orient returns
// them): the recursion of orc_kclique without the orientation step, so that a
// sample of a large graph can be timed on its own.
uint64_t orc_kclique_dag_ranges(int64_t n, const int64_t* off, const int32_t* adj, int k, const int64_t* ranges,
                                int64_t n_ranges) {
    Dag g;
    g.off.assign(off, off + n + 1);
    g.adj.assign(adj, adj + off[n]);
    const int64_t m = off[n];
    uint64_t total = 0;
    for (int64_t r = 0; r < n_ranges; ++r) {
        const int64_t lo = ranges[2 * r], hi = ranges[2 * r + 1];
        int64_t u = 0;
        for (int64_t p = lo; p < hi && p < m; ++p) {
            while (g.off[u + 1] <= p) ++u;
            int32_t v = g.adj[p];
            std::vector<int32_t> C = intersect(g.adj.data() + g.off[u], g.off[u + 1] - g.off[u],
                                               g.adj.data() + g.off[v], g.off[v + 1] - g.off[v]);
            if (k == 3) total += C.size();
            else if ((int)C.size() >= k - 2) total += count_in(g, C, k - 2);
        }
    }
    return total;
}

// ---------------------------------------------------------------------------
// k-clique counting by pivoting (Sec. 6.4.2, the second algorithm of the
// k-clique study; Jain and Seshadhri's succinct clique tree).  For every DAG
// edge (u, v) the candidate set is S = N+(u) n N+(v) with u and v "held".
// A node (S, h held, p pivots) with S empty is a leaf and stands for the
// cliques made of its held vertices plus any subset of its pivots: it adds
// C(p, k - h) k-cliques.  Otherwise the pivot x is the vertex of S with the
// most neighbours inside S (ties: the smallest id); the branches are the
// vertices w of S not adjacent to x (x itself first among them, in S's order);
// branch i recurses on S n N(w_i) minus the earlier branch vertices, with w_i
// counted as a pivot when it is x and as held otherwise.  N is the undirected
// neighbourhood.  Every k-clique is counted once; the recursion depth is
// bounded by the pivots, so the search is shallow compared with orientation.
static uint64_t binom_u64(uint64_t n, int r) {
    if (r < 0 || (uint64_t)r > n) return 0;
    unsigned __int128 c = 1;
    for (int i = 1; i <= r; ++i) c = c * (n - (uint64_t)r + (uint64_t)i) / (uint64_t)i;
    return (uint64_t)c;
}

struct UndirectedCsr { std::vector<int64_t> off; std::vector<int32_t> adj; };

static UndirectedCsr undirected(int64_t n, const int32_t* edges, int64_t m) {
    UndirectedCsr g;
    g.off.assign(n + 1, 0);
    for (int64_t e = 0; e < m; ++e) { ++g.off[edges[2 * e] + 1]; ++g.off[edges[2 * e + 1] + 1]; }
    for (int64_t v = 0; v < n; ++v) g.off[v + 1] += g.off[v];
    g.adj.assign(2 * m, 0);
    std::vector<int64_t> fill(g.off.begin(), g.off.end() - 1);
    for (int64_t e = 0; e < m; ++e) {
        g.adj[fill[edges[2 * e]]++] = edges[2 * e + 1];
        g.adj[fill[edges[2 * e + 1]]++] = edges[2 * e];
    }
    for (int64_t v = 0; v < n; ++v) std::sort(g.adj.begin() + g.off[v], g.adj.begin() + g.off[v + 1]);
    return g;
}

static uint64_t pivot_count(const UndirectedCsr& g, const std::vector<int32_t>& S, int h, int p, int k,
                            uint64_t* nodes) {
    ++*nodes;
    if (h > k) return 0;
    if (S.empty()) return binom_u64((uint64_t)p, k - h);
    // the pivot: most neighbours inside S, the smallest id on ties (S is sorted by id)
    int32_t x = S[0];
    size_t best = 0;
    bool first = true;
    for (int32_t y : S) {
        std::vector<int32_t> t = intersect(g.adj.data() + g.off[y], g.off[y + 1] - g.off[y], S.data(), (int64_t)S.size());
        if (first || t.size() > best) { best = t.size(); x = y; first = false; }
    }
    std::vector<int32_t> nx = intersect(g.adj.data() + g.off[x], g.off[x + 1] - g.off[x], S.data(), (int64_t)S.size());
    // branch vertices: x, then the vertices of S not adjacent to x, in S's order
    std::vector<int32_t> branch{x};
    for (int32_t y : S)
        if (y != x && !std::binary_search(nx.begin(), nx.end(), y)) branch.push_back(y);
    uint64_t total = 0;
    std::vector<int32_t> done;   // earlier branch vertices, kept sorted
    for (int32_t w : branch) {
        std::vector<int32_t> nw = intersect(g.adj.data() + g.off[w], g.off[w + 1] - g.off[w], S.data(), (int64_t)S.size());
        std::vector<int32_t> Sw;
        std::set_difference(nw.begin(), nw.end(), done.begin(), done.end(), std::back_inserter(Sw));
        total += (w == x) ? pivot_count(g, Sw, h, p + 1, k, nodes) : pivot_count(g, Sw, h + 1, p, k, nodes);
        done.insert(std::upper_bound(done.begin(), done.end(), w), w);
    }
    return total;
}

// The same recursion counting every clique size at once: a leaf (h, p) adds
// C(p, j - h) to count[j] for every j (the pivot search does not depend on k,
// only the pruning h > k does, which the all-sizes form leaves out).  It runs
// on the subgraph induced by the edge's candidate set C: nbr[a] lists the
// members of C adjacent to member a (local indices in C's id order, so the
// smallest-id tie rule is the smallest index), found from the members' DAG
// out-lists and mirrored.
static void pivot_all_induced(const std::vector<std::vector<int32_t>>& nbr, const std::vector<int32_t>& S, int h, int p,
                              int kmax, uint64_t* count) {
    if (h > kmax) return;
    if (S.empty()) {
        for (int j = h; j <= kmax && j - h <= p; ++j) count[j] += binom_u64((uint64_t)p, j - h);
        return;
    }
    int32_t x = S[0];
    size_t best = 0;
    bool first = true;
    for (int32_t y : S) {
        std::vector<int32_t> t = intersect(nbr[y].data(), (int64_t)nbr[y].size(), S.data(), (int64_t)S.size());
        if (first || t.size() > best) { best = t.size(); x = y; first = false; }
    }
    std::vector<int32_t> nx = intersect(nbr[x].data(), (int64_t)nbr[x].size(), S.data(), (int64_t)S.size());
    std::vector<int32_t> branch{x};
    for (int32_t y : S)
        if (y != x && !std::binary_search(nx.begin(), nx.end(), y)) branch.push_back(y);
    std::vector<int32_t> done;
    for (int32_t w : branch) {
        std::vector<int32_t> nw = intersect(nbr[w].data(), (int64_t)nbr[w].size(), S.data(), (int64_t)S.size());
        std::vector<int32_t> Sw;
        std::set_difference(nw.begin(), nw.end(), done.begin(), done.end(), std::back_inserter(Sw));
        if (w == x) pivot_all_induced(nbr, Sw, h, p + 1, kmax, count);
        else pivot_all_induced(nbr, Sw, h + 1, p, kmax, count);
        done.insert(std::upper_bound(done.begin(), done.end(), w), w);
    }
}

// The undirected CSR (sorted lists) of a graph, for the all-sizes count below.
void orc_undirected(int64_t n, const int32_t* edges, int64_t m, int64_t* uoff, int32_t* uadj) {
    UndirectedCsr g = undirected(n, edges, m);
    std::memcpy(uoff, g.off.data(), (n + 1) * sizeof(int64_t));
    std::memcpy(uadj, g.adj.data(), 2 * m * sizeof(int32_t));
}

// Clique counts of every size 3 .. kmax by pivoting, over the DAG edges of the
// given ranges of a graph already oriented (off/adj as orc_orient returns them)
// with its undirected CSR (uoff/uadj as orc_undirected returns them):
// count[j] for j = 0 .. kmax (entries below 3 stay 0).
void orc_kclique_pivot_all(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* ranges, int64_t n_ranges,
                           int kmax, uint64_t* count) {
    for (int j = 0; j <= kmax; ++j) count[j] = 0;
    const int64_t m = off[n];
    std::vector<uint64_t> c(kmax + 1, 0);
    for (int64_t r = 0; r < n_ranges; ++r) {
        int64_t u = 0;
        for (int64_t e = ranges[2 * r]; e < ranges[2 * r + 1] && e < m; ++e) {
            while (off[u + 1] <= e) ++u;
            const int32_t v = adj[e];
            std::vector<int32_t> C = intersect(adj + off[u], off[u + 1] - off[u], adj + off[v], off[v + 1] - off[v]);
            // the subgraph induced by C, in local indices
            std::vector<std::vector<int32_t>> nbr(C.size());
            for (size_t a = 0; a < C.size(); ++a) {
                const int32_t y = C[a];
                std::vector<int32_t> out = intersect(adj + off[y], off[y + 1] - off[y], C.data(), (int64_t)C.size());
                for (int32_t z : out) {
                    const int32_t b = (int32_t)(std::lower_bound(C.begin(), C.end(), z) - C.begin());
                    nbr[a].push_back(b);
                    nbr[b].push_back((int32_t)a);
                }
            }
            for (auto& l : nbr) std::sort(l.begin(), l.end());
            std::vector<int32_t> S(C.size());
            for (size_t a = 0; a < C.size(); ++a) S[a] = (int32_t)a;
            pivot_all_induced(nbr, S, 2, 0, kmax, c.data());
        }
    }
    for (int j = 3; j <= kmax; ++j) count[j] = c[j];
}

// Total k-clique count by pivoting over the DAG edges [lo, hi) of the
// (degree, id) orientation (all edges: lo = 0, hi = m); *nodes (optional)
// receives the number of recursion nodes.
uint64_t orc_kclique_pivot(int64_t n, const int32_t* edges, int64_t m, int k, int64_t lo, int64_t hi, uint64_t* nodes) {
    if (k < 3) return 0;
    Dag d = orient(n, edges, m, 0);
    UndirectedCsr g = undirected(n, edges, m);
    uint64_t total = 0, nd = 0;
    int64_t u = 0;
    for (int64_t e = lo; e < hi && e < m; ++e) {
        while (d.off[u + 1] <= e) ++u;
        const int32_t v = d.adj[e];
        std::vector<int32_t> C = intersect(d.adj.data() + d.off[u], d.off[u + 1] - d.off[u], d.adj.data() + d.off[v],
                                           d.off[v + 1] - d.off[v]);
        total += pivot_count(g, C, 2, 0, k, &nd);
    }
    if (nodes) *nodes = nd;
    return total;
}

// The oriented DAG itself (CSR), for checking the GPU orientation step.
// off has n+1 entries, adj has m entries.
void orc_orient(int64_t n, const int32_t* edges, int64_t m, int order_mode, int64_t* off, int32_t* adj) {
    Dag g = orient(n, edges, m, order_mode);
    std::memcpy(off, g.off.data(), (n + 1) * sizeof(int64_t));
    std::memcpy(adj, g.adj.data(), m * sizeof(int32_t));
}

// Brute force for tiny graphs (n <= 64): every k-subset of the vertices in
// lexicographic order, kept if all of its pairs are edges.
uint64_t orc_kclique_brute(int n, const int32_t* edges, int64_t m, int k) {
    std::vector<std::vector<char>> a(n, std::vector<char>(n, 0));
    for (int64_t e = 0; e < m; ++e) {
        a[edges[2 * e]][edges[2 * e + 1]] = 1;
        a[edges[2 * e + 1]][edges[2 * e]] = 1;
    }
    if (k <= 0 || k > n) return k == 0 ? 1 : 0;
    std::vector<int> c(k);
    for (int i = 0; i < k; ++i) c[i] = i;
    uint64_t count = 0;
    while (true) {
        bool clique = true;
        for (int i = 0; i < k && clique; ++i)
            for (int j = i + 1; j < k && clique; ++j)
                if (!a[c[i]][c[j]]) clique = false;
        if (clique) ++count;
        int i = k - 1;
        while (i >= 0 && c[i] == n - k + i) --i;
        if (i < 0) break;
        ++c[i];
        for (int j = i + 1; j < k; ++j) c[j] = c[j - 1] + 1;
    }
    return count;
}

// ---------------------------------------------------------------------------
// Full binary task tree microbenchmark (Sec. 6.1, Sec. 6.2).  Node v has the
// children 2v and 2v+1; the leaves are the nodes of level D.  A leaf's
// function index is the high half of splitmix64(v) reduced mod K, and its value
// is the sum, mod 2^64, of its function over the inputs (v << 32) + i for
// i = 0 .. iters-1.  The four functions, as the program definition states them:
//   f0: multiply by 0x9E3779B97F4A7C15, xor the value shifted right 29, multiply
//       by 0xBF58476D1CE4E5B9, xor the value shifted right 32;
//   f1: xor x shifted left 13, then xor shifted right 7, then xor shifted left 17,
//       multiply by 0x2545F4914F6CDD1D;
//   f2: add 0x632BE59BD9B4E019, multiply by 0x94D049BB133111EB, rotate left 23
//       and xor with the value shifted right 11;
//   f3: xor x with x shifted right 32, multiply by 0xD6E8FEB86659FD93, xor the
//       value shifted right 28.
// The serial elision sums the two subtrees; a block-mode cutoff c only changes
// how many tasks are created (a node c levels above the leaves is one task).
static uint64_t bt_fn(int k, uint64_t x) {
    uint64_t z;
    if (k == 0) {
        z = x * 0x9E3779B97F4A7C15ULL;
        z = z ^ (z >> 29);
        z = z * 0xBF58476D1CE4E5B9ULL;
        return z ^ (z >> 32);
    }
    if (k == 1) {
        z = x ^ (x << 13);
        z = z ^ (z >> 7);
        z = z ^ (z << 17);
        return z * 0x2545F4914F6CDD1DULL;
    }
    if (k == 2) {
        z = (x + 0x632BE59BD9B4E019ULL) * 0x94D049BB133111EBULL;
        uint64_t rotated = (z << 23) | (z >> 41);
        return rotated ^ (z >> 11);
    }
    z = x ^ (x >> 32);
    z = z * 0xD6E8FEB86659FD93ULL;
    return z ^ (z >> 28);
}

static uint64_t bt_leaf(uint64_t v, int iters, int K) {
    int k = 0;
    if (K > 1) k = (int)((splitmix64(v) >> 32) % (uint64_t)K);
    uint64_t sum = 0;
    for (int i = 0; i < iters; ++i) sum += bt_fn(k, (v << 32) + (uint64_t)i);
    return sum;
}

static uint64_t bt_rec(uint64_t v, int level, int D, int iters, int K, int cutoff, uint64_t* tasks) {
    // a block-mode task that runs its whole subtree counts once
    bool whole = level == D || (cutoff > 0 && D - level <= cutoff);
    *tasks += 1;
    if (whole) {
        uint64_t s = 0;
        uint64_t first = v << (D - level), n = 1ULL << (D - level);
        for (uint64_t j = 0; j < n; ++j) s += bt_leaf(first + j, iters, K);
        return s;
    }
    return bt_rec(2 * v, level + 1, D, iters, K, cutoff, tasks) + bt_rec(2 * v + 1, level + 1, D, iters, K, cutoff, tasks);
}

uint64_t orc_bintree(int depth, int iters, int K, int cutoff, uint64_t* tasks) {
    uint64_t t = 0;
    uint64_t r = bt_rec(1, 0, depth, iters, K, cutoff, &t);
    if (tasks) *tasks = t;
    return r;
}

uint64_t orc_bintree_leaf(uint64_t v, int iters, int K) { return bt_leaf(v, iters, K); }

}  // extern "C"
