// CPU oracle for the Laplace FMM pipeline (Sec. 6.4.1) -- TEST INFRASTRUCTURE ONLY.
//
// The plain definition is phi_i = sum_{j != i} q_j / |x_i - x_j|; the FMM
// approximates it, so this oracle runs the same algorithm in FP64, step by
// step, in the order the pipeline names: octree construction, upward pass
// (P2M, M2M), dual-tree traversal building the M2L and P2P lists, then M2L,
// downward pass (L2L, L2P) and P2P.  Choices the paper leaves open, fixed
// here and in the GPU code alike:
//   * Tree: the bounding cube of the points (side = largest extent, centred);
//     points get 21-bit-per-axis Morton codes q = min(2^21-1, floor((x-lo)*2^21/side))
//     and are ordered by (code, index); a cell splits into its non-empty
//     octants (Morton order) while it holds more than leaf_size points and its
//     level is below 21.  Cells are numbered breadth first.
//   * Expansions: Cartesian Taylor about the geometric cell centre, total
//     order p.  M_a = sum_j q_j (x_j - c)^a; L_b = sum_a (-1)^|a| C(a+b, b)
//     T_{a+b}(t - s) M_a with |a| + |b| <= p, where T_n = d^n(1/r)/n! from the
//     recurrence |n| r^2 T_n = -(2|n|-1) sum_i x_i T_{n-e_i} - (|n|-1) sum_i T_{n-2e_i}.
//   * MAC: a pair (A, B) is accepted iff (R_A + R_B)^2 < theta^2 |c_A - c_B|^2,
//     R = half-diagonal of the cell cube.  Accepted -> M2L(A <- B); two
//     leaves -> P2P(A <- B); a self pair splits into all child pairs; else the
//     larger cell splits (equal size: both).
// Parity status: pinned (exact at N <= leaf size, theta -> 0 gives the direct
// sum, the error falls as p grows; see tests/test_oracle_pins.py).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

struct MI { int a, b, c; };

// multi-indices of total degree <= p, ordered by degree, then a desc, then b desc
std::vector<MI> multi_indices(int p) {
    std::vector<MI> v;
    for (int k = 0; k <= p; ++k)
        for (int a = k; a >= 0; --a)
            for (int b = k - a; b >= 0; --b) v.push_back({a, b, k - a - b});
    return v;
}

// Pascal's triangle, C(n, k) for n <= 16
struct Binomials {
    double c[17][17];
    Binomials() {
        for (int n = 0; n <= 16; ++n)
            for (int k = 0; k <= 16; ++k) c[n][k] = (k == 0) ? 1.0 : (n == 0 ? 0.0 : c[n - 1][k - 1] + c[n - 1][k]);
    }
};
const Binomials kBinom;
double binom(int n, int k) { return (k < 0 || k > n) ? 0.0 : kBinom.c[n][k]; }

double ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

struct Expansion {
    int p;
    std::vector<MI> mi;
    std::vector<int> index;   // (a, b, c) -> position, table of (p+1)^3
    std::vector<size_t> upto; // upto[k] = number of multi-indices of degree <= k (they come first)
    explicit Expansion(int p_) : p(p_), mi(multi_indices(p_)), index((p_ + 1) * (p_ + 1) * (p_ + 1), -1), upto(p_ + 1) {
        for (size_t i = 0; i < mi.size(); ++i) index[(mi[i].a * (p + 1) + mi[i].b) * (p + 1) + mi[i].c] = (int)i;
        for (int k = 0; k <= p; ++k) upto[k] = (size_t)((k + 1) * (k + 2) * (k + 3) / 6);
    }
    int at(int a, int b, int c) const {
        if (a < 0 || b < 0 || c < 0 || a + b + c > p) return -1;
        return index[(a * (p + 1) + b) * (p + 1) + c];
    }
    // T_n(r) = d^n (1/|r|) / n!  for |n| <= p
    void derivatives(double x, double y, double z, std::vector<double>& T) const {
        const double r2 = x * x + y * y + z * z;
        T.assign(mi.size(), 0.0);
        T[0] = 1.0 / std::sqrt(r2);
        for (size_t i = 1; i < mi.size(); ++i) {
            const MI& n = mi[i];
            const int k = n.a + n.b + n.c;
            double s = 0.0;
            if (n.a > 0) s += x * T[at(n.a - 1, n.b, n.c)];
            if (n.b > 0) s += y * T[at(n.a, n.b - 1, n.c)];
            if (n.c > 0) s += z * T[at(n.a, n.b, n.c - 1)];
            double s2 = 0.0;
            if (n.a > 1) s2 += T[at(n.a - 2, n.b, n.c)];
            if (n.b > 1) s2 += T[at(n.a, n.b - 2, n.c)];
            if (n.c > 1) s2 += T[at(n.a, n.b, n.c - 2)];
            T[i] = (-(2.0 * k - 1.0) * s - (k - 1.0) * s2) / (k * r2);
        }
    }
};

struct Cell {
    int level;
    uint64_t ix, iy, iz;       // integer cube coordinates at this level
    double cx, cy, cz, h;      // centre and half side
    int64_t first, count;      // range of sorted points
    int64_t child_first;       // index of the first child, -1 for a leaf
    int nchild;
    int64_t parent;            // -1 for the root
};

uint64_t spread21(uint64_t v) {
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
}

struct Tree {
    double lo[3], side;
    std::vector<int64_t> order;   // sorted position -> input index
    std::vector<uint64_t> code;   // sorted codes
    std::vector<Cell> cells;
};

Tree build_tree(int64_t n, const double* pos, int leaf_size) {
    Tree t;
    double mn[3], mx[3];
    for (int d = 0; d < 3; ++d) { mn[d] = pos[d]; mx[d] = pos[d]; }
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) { mn[d] = std::min(mn[d], pos[3 * i + d]); mx[d] = std::max(mx[d], pos[3 * i + d]); }
    double side = 0.0;
    for (int d = 0; d < 3; ++d) side = std::max(side, mx[d] - mn[d]);
    if (side <= 0.0) side = 1.0;
    t.side = side;
    for (int d = 0; d < 3; ++d) t.lo[d] = (mn[d] + mx[d]) * 0.5 - side * 0.5;
    const double scale = 2097152.0 / side;
    std::vector<uint64_t> codes(n);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t q[3];
        for (int d = 0; d < 3; ++d) {
            double f = std::floor((pos[3 * i + d] - t.lo[d]) * scale);
            if (f < 0.0) f = 0.0;
            if (f > 2097151.0) f = 2097151.0;
            q[d] = (uint64_t)f;
        }
        codes[i] = spread21(q[0]) | (spread21(q[1]) << 1) | (spread21(q[2]) << 2);
    }
    t.order.resize(n);
    std::iota(t.order.begin(), t.order.end(), 0);
    std::sort(t.order.begin(), t.order.end(), [&](int64_t a, int64_t b) {
        return codes[a] != codes[b] ? codes[a] < codes[b] : a < b;
    });
    t.code.resize(n);
    for (int64_t i = 0; i < n; ++i) t.code[i] = codes[t.order[i]];
    Cell root{0, 0, 0, 0, t.lo[0] + side * 0.5, t.lo[1] + side * 0.5, t.lo[2] + side * 0.5, side * 0.5, 0, n, -1, 0, -1};
    t.cells.push_back(root);
    size_t level_begin = 0;
    while (level_begin < t.cells.size()) {
        const size_t level_end = t.cells.size();
        for (size_t ci = level_begin; ci < level_end; ++ci) {
            Cell c = t.cells[ci];
            if (c.count <= leaf_size || c.level >= 21) continue;
            const int shift = 3 * (20 - c.level);
            int64_t s = c.first;
            const int64_t e = c.first + c.count;
            t.cells[ci].child_first = (int64_t)t.cells.size();
            int nch = 0;
            for (int o = 0; o < 8; ++o) {
                int64_t k = s;
                while (k < e && (int)((t.code[k] >> shift) & 7ull) == o) ++k;
                if (k > s) {
                    Cell ch;
                    ch.level = c.level + 1;
                    ch.ix = 2 * c.ix + (o & 1);
                    ch.iy = 2 * c.iy + ((o >> 1) & 1);
                    ch.iz = 2 * c.iz + ((o >> 2) & 1);
                    const double cell = side / (double)(1ull << ch.level);
                    ch.cx = t.lo[0] + ((double)ch.ix + 0.5) * cell;
                    ch.cy = t.lo[1] + ((double)ch.iy + 0.5) * cell;
                    ch.cz = t.lo[2] + ((double)ch.iz + 0.5) * cell;
                    ch.h = cell * 0.5;
                    ch.first = s;
                    ch.count = k - s;
                    ch.child_first = -1;
                    ch.nchild = 0;
                    ch.parent = (int64_t)ci;
                    t.cells.push_back(ch);
                    ++nch;
                }
                s = k;
            }
            t.cells[ci].nchild = nch;
        }
        level_begin = level_end;
    }
    return t;
}

const double kSqrt3 = 1.7320508075688772;

bool mac(const Cell& A, const Cell& B, double theta) {
    const double dx = A.cx - B.cx, dy = A.cy - B.cy, dz = A.cz - B.cz;
    const double d2 = (dx * dx + dy * dy) + dz * dz;
    const double R = A.h * kSqrt3 + B.h * kSqrt3;
    return R * R < (theta * theta) * d2;
}

void traverse(const Tree& t, int64_t a, int64_t b, double theta, std::vector<int64_t>& m2l, std::vector<int64_t>& p2p) {
    const Cell& A = t.cells[a];
    const Cell& B = t.cells[b];
    if (a != b && mac(A, B, theta)) { m2l.push_back(a); m2l.push_back(b); return; }
    const bool la = A.child_first < 0, lb = B.child_first < 0;
    if (la && lb) { p2p.push_back(a); p2p.push_back(b); return; }
    const bool split_a = !la && (lb || A.level <= B.level);
    const bool split_b = !lb && (la || B.level <= A.level);
    if (split_a && split_b) {
        for (int i = 0; i < A.nchild; ++i)
            for (int j = 0; j < B.nchild; ++j) traverse(t, A.child_first + i, B.child_first + j, theta, m2l, p2p);
    } else if (split_a) {
        for (int i = 0; i < A.nchild; ++i) traverse(t, A.child_first + i, b, theta, m2l, p2p);
    } else {
        for (int j = 0; j < B.nchild; ++j) traverse(t, a, B.child_first + j, theta, m2l, p2p);
    }
}

}  // namespace

extern "C" {

// Full FP64 FMM.  With targets == NULL, phi (n, input order) receives every
// potential; otherwise phi[k] is the potential at point targets[k], and the
// downward pass (M2L, L2L, L2P, P2P) is restricted to the cells that contain
// a target (the same arithmetic for those points).  Optional outputs: list
// lengths and the lists themselves (pairs of cell indices).
int orc_fmm(int64_t n, const double* pos, const double* q, int p, double theta, int leaf_size,
            const int64_t* targets, int64_t n_targets, double* phi,
            int64_t* n_cells, int64_t* n_m2l, int64_t* n_p2p, int64_t* m2l_out, int64_t m2l_cap, int64_t* p2p_out,
            int64_t p2p_cap) {
    if (p < 0 || p > 8 || n < 1 || leaf_size < 1) return 1;
    Tree t = build_tree(n, pos, leaf_size);
    Expansion E(p);
    const size_t nt = E.mi.size();
    const int64_t nc = (int64_t)t.cells.size();
    // cells whose local expansion is needed: every cell when all points are
    // targets, else the leaves holding a target and their ancestors
    std::vector<char> wanted(nc, targets ? 0 : 1), is_target(n, targets ? 0 : 1);
    if (targets) {
        std::vector<int64_t> pos_of(n), leaf_of(n);
        for (int64_t k = 0; k < n; ++k) pos_of[t.order[k]] = k;
        for (int64_t ci = 0; ci < nc; ++ci)
            if (t.cells[ci].child_first < 0)
                for (int64_t k = t.cells[ci].first; k < t.cells[ci].first + t.cells[ci].count; ++k) leaf_of[k] = ci;
        for (int64_t k = 0; k < n_targets; ++k) {
            if (targets[k] < 0 || targets[k] >= n) return 1;
            is_target[targets[k]] = 1;
            for (int64_t c = leaf_of[pos_of[targets[k]]]; c >= 0; c = t.cells[c].parent) wanted[c] = 1;
        }
    }
    std::vector<double> M(nc * nt, 0.0), L(nc * nt, 0.0);
    // upward pass: P2M at leaves, M2M from children (deepest cells first)
    for (int64_t ci = nc - 1; ci >= 0; --ci) {
        const Cell& c = t.cells[ci];
        double* m = &M[ci * nt];
        if (c.child_first < 0) {
            for (int64_t k = c.first; k < c.first + c.count; ++k) {
                const int64_t j = t.order[k];
                const double dx = pos[3 * j] - c.cx, dy = pos[3 * j + 1] - c.cy, dz = pos[3 * j + 2] - c.cz;
                for (size_t a = 0; a < nt; ++a)
                    m[a] += q[j] * ipow(dx, E.mi[a].a) * ipow(dy, E.mi[a].b) * ipow(dz, E.mi[a].c);
            }
        } else {
            for (int ch = 0; ch < c.nchild; ++ch) {
                const Cell& d = t.cells[c.child_first + ch];
                const double* md = &M[(c.child_first + ch) * nt];
                const double sx = d.cx - c.cx, sy = d.cy - c.cy, sz = d.cz - c.cz;
                for (size_t a = 0; a < nt; ++a) {
                    const MI& al = E.mi[a];
                    double acc = 0.0;
                    for (size_t b = 0; b < E.upto[al.a + al.b + al.c]; ++b) {
                        const MI& be = E.mi[b];
                        if (be.a > al.a || be.b > al.b || be.c > al.c) continue;
                        acc += binom(al.a, be.a) * binom(al.b, be.b) * binom(al.c, be.c) * ipow(sx, al.a - be.a) *
                               ipow(sy, al.b - be.b) * ipow(sz, al.c - be.c) * md[b];
                    }
                    m[a] += acc;
                }
            }
        }
    }
    // dual-tree traversal
    std::vector<int64_t> m2l, p2p;
    traverse(t, 0, 0, theta, m2l, p2p);
    // M2L
    std::vector<double> T;
    for (size_t k = 0; k < m2l.size(); k += 2) {
        if (!wanted[m2l[k]]) continue;
        const Cell& A = t.cells[m2l[k]];
        const Cell& B = t.cells[m2l[k + 1]];
        E.derivatives(A.cx - B.cx, A.cy - B.cy, A.cz - B.cz, T);
        const double* mb = &M[m2l[k + 1] * nt];
        double* la = &L[m2l[k] * nt];
        for (size_t b = 0; b < nt; ++b) {
            const MI& be = E.mi[b];
            double acc = 0.0;
            for (size_t a = 0; a < E.upto[p - (be.a + be.b + be.c)]; ++a) {  // |a| + |b| <= p
                const MI& al = E.mi[a];
                const int s = al.a + al.b + al.c;
                const double sign = (s & 1) ? -1.0 : 1.0;
                const double cab = binom(al.a + be.a, be.a) * binom(al.b + be.b, be.b) * binom(al.c + be.c, be.c);
                acc += sign * cab * T[E.at(al.a + be.a, al.b + be.b, al.c + be.c)] * mb[a];
            }
            la[b] += acc;
        }
    }
    // downward pass: L2L parent -> children (breadth first), L2P at leaves
    std::vector<double> out(n, 0.0);
    for (int64_t ci = 0; ci < nc; ++ci) {
        if (!wanted[ci]) continue;
        const Cell& c = t.cells[ci];
        const double* lc = &L[ci * nt];
        if (c.child_first >= 0) {
            for (int ch = 0; ch < c.nchild; ++ch) {
                const Cell& d = t.cells[c.child_first + ch];
                double* ld = &L[(c.child_first + ch) * nt];
                const double sx = d.cx - c.cx, sy = d.cy - c.cy, sz = d.cz - c.cz;
                for (size_t g = 0; g < nt; ++g) {
                    const MI& ga = E.mi[g];
                    double acc = 0.0;
                    for (size_t b = 0; b < nt; ++b) {
                        const MI& be = E.mi[b];
                        if (be.a < ga.a || be.b < ga.b || be.c < ga.c) continue;
                        acc += binom(be.a, ga.a) * binom(be.b, ga.b) * binom(be.c, ga.c) * ipow(sx, be.a - ga.a) *
                               ipow(sy, be.b - ga.b) * ipow(sz, be.c - ga.c) * lc[b];
                    }
                    ld[g] += acc;
                }
            }
        } else {
            for (int64_t k = c.first; k < c.first + c.count; ++k) {
                const int64_t i = t.order[k];
                if (!is_target[i]) continue;
                const double dx = pos[3 * i] - c.cx, dy = pos[3 * i + 1] - c.cy, dz = pos[3 * i + 2] - c.cz;
                double acc = 0.0;
                for (size_t b = 0; b < nt; ++b)
                    acc += lc[b] * ipow(dx, E.mi[b].a) * ipow(dy, E.mi[b].b) * ipow(dz, E.mi[b].c);
                out[i] += acc;
            }
        }
    }
    // P2P
    for (size_t k = 0; k < p2p.size(); k += 2) {
        if (!wanted[p2p[k]]) continue;
        const Cell& A = t.cells[p2p[k]];
        const Cell& B = t.cells[p2p[k + 1]];
        for (int64_t x = A.first; x < A.first + A.count; ++x) {
            const int64_t i = t.order[x];
            if (!is_target[i]) continue;
            double acc = 0.0;
            for (int64_t y = B.first; y < B.first + B.count; ++y) {
                const int64_t j = t.order[y];
                if (i == j) continue;
                const double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                             dz = pos[3 * i + 2] - pos[3 * j + 2];
                acc += q[j] / std::sqrt(dx * dx + dy * dy + dz * dz);
            }
            out[i] += acc;
        }
    }
    if (targets)
        for (int64_t k = 0; k < n_targets; ++k) phi[k] = out[targets[k]];
    else
        std::memcpy(phi, out.data(), n * sizeof(double));
    if (n_cells) *n_cells = nc;
    if (n_m2l) *n_m2l = (int64_t)m2l.size() / 2;
    if (n_p2p) *n_p2p = (int64_t)p2p.size() / 2;
    if (m2l_out) std::memcpy(m2l_out, m2l.data(), std::min<int64_t>(m2l_cap * 2, (int64_t)m2l.size()) * sizeof(int64_t));
    if (p2p_out) std::memcpy(p2p_out, p2p.data(), std::min<int64_t>(p2p_cap * 2, (int64_t)p2p.size()) * sizeof(int64_t));
    return 0;
}

// The tree alone: cell records as 8 doubles each (level, first, count, child_first,
// nchild, cx, cy, cz) and the sorted order; returns the number of cells.
int64_t orc_fmm_tree(int64_t n, const double* pos, int leaf_size, double* cells_out, int64_t cap, int64_t* order_out) {
    Tree t = build_tree(n, pos, leaf_size);
    const int64_t nc = (int64_t)t.cells.size();
    for (int64_t i = 0; i < nc && i < cap; ++i) {
        const Cell& c = t.cells[i];
        double* r = cells_out + 8 * i;
        r[0] = c.level; r[1] = (double)c.first; r[2] = (double)c.count; r[3] = (double)c.child_first;
        r[4] = c.nchild; r[5] = c.cx; r[6] = c.cy; r[7] = c.cz;
    }
    if (order_out) std::memcpy(order_out, t.order.data(), n * sizeof(int64_t));
    return nc;
}

// Taylor coefficients T_n(r) = d^n(1/|r|)/n! for |n| <= p, in the expansion's
// multi-index order (degree, then a descending, then b descending).
int orc_taylor(int p, double x, double y, double z, double* out) {
    if (p < 0 || p > 12) return 1;
    Expansion E(p);
    std::vector<double> T;
    E.derivatives(x, y, z, T);
    std::memcpy(out, T.data(), T.size() * sizeof(double));
    return 0;
}

// Direct sum for selected targets: phi_i = sum_{j != i} q_j / |x_i - x_j|.
void orc_direct(int64_t n, const double* pos, const double* q, const int64_t* targets, int64_t nt, double* out) {
    for (int64_t k = 0; k < nt; ++k) {
        const int64_t i = targets[k];
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1], dz = pos[3 * i + 2] - pos[3 * j + 2];
            acc += q[j] / std::sqrt(dx * dx + dy * dy + dz * dz);
        }
        out[k] = acc;
    }
}

}  // extern "C"
