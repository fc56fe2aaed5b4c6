// Internal layout of the Laplace FMM pipeline (Sec. 6.4.1): cell records,
// expansion tables and the traversal environment shared by the tree build,
// the dual-tree traversal task program and the evaluation kernels.
//
// Cells are numbered breadth first (level, then Morton order), so the cells
// of level l are the index range [lstart[l], lstart[l+1]).  Per cell:
//   geom  Dbl4 {cx, cy, cz, h}   centre and half side of the cell cube
//   info  int4    {first, count, child_first (-1 for a leaf), level << 8 | nchild}
// Points are kept in Morton order: pts[k] = {x, y, z, q} of input point order[k].
// Expansions are Cartesian Taylor series of total order p about the cell
// centre, nt = (p+1)(p+2)(p+3)/6 coefficients per cell, stored in FP64 in the
// multi-index order (degree, then a descending, then b descending).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "gtap.h"

namespace gtap {
namespace fmm {

struct __align__(32) Dbl4 {
    double x, y, z, w;
};
__host__ __device__ inline Dbl4 make_dbl4(double x, double y, double z, double w) {
    Dbl4 v;
    v.x = x; v.y = y; v.z = z; v.w = w;
    return v;
}

constexpr int kMaxOrder = 8;
constexpr int kMaxCoef = (kMaxOrder + 1) * (kMaxOrder + 2) * (kMaxOrder + 3) / 6;   // 165
constexpr int kMaxLevel = 21;          // 21 bits per axis in the Morton codes
constexpr int kMaxLeaf = 64;
constexpr double kSqrt3 = 1.7320508075688772;

__host__ __device__ constexpr int n_coef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// Traversal constants kept in device memory (the plan's, refreshed before every traversal).
//  screen: the MAC may first be decided in FP32 from the exact lattice centres
//  (3 (h_A + h_B)^2 against theta^2 |d|^2 in lattice units); only a pair within
//  the relative margin of the boundary takes the FP64 test that reproduces the
//  oracle's rounding.  The margin (1e-5) exceeds the FP32 error (< 4e-7) plus
//  the gap between exact and FP64-rounded centres, which the host bounds from
//  the coordinates' magnitude and disables screening when it is not small.
struct DttAux {
    double theta;
    float theta2, margin;
    long long m2l_cap, p2p_cap;      // list capacities (entries)
    int screen, pad;
};

// Read-only environment of one traversal (lives in the root's 64-byte env).
struct DttEnv {
    const Dbl4* geom;
    const int4* info;
    const int4* lat;                 // lattice centres: (2i+1) << (21 - level) per axis, level
    unsigned long long* m2l;         // (target << 32 | source) entries
    unsigned long long* p2p;
    unsigned long long* counters;    // [0] M2L appends, [1] P2P appends (may exceed the capacities)
    const DttAux* aux;
    int n_cells, pad;
};
static_assert(sizeof(DttEnv) == 64, "DttEnv must fill the root environment");

// Pairs carried by one traversal task (payload of a 128-byte record).
constexpr int kDttGroup = 13;
struct DttSpawn {
    uint32_t root, n;
    unsigned long long pr[kDttGroup];
};
static_assert(sizeof(DttSpawn) == 112, "DttSpawn must fill a 128-byte record payload");

// Expansion tables, built on the host for one order p (device copies).
//  deriv[i], i >= 1: indices of n - e_x, n - e_y, n - e_z and n - 2e_x, n - 2e_y,
//    n - 2e_z (or -1) and k = |n|, for the recurrence of the Taylor coefficients
//    of 1/r: |n| r^2 T_n = -(2|n|-1) sum_d x_d T_{n-e_d} - (|n|-1) sum_d T_{n-2e_d}.
//  m2l terms, grouped by beta: (alpha, alpha+beta) with |alpha| + |beta| <= p and
//    coefficient (-1)^|alpha| C(alpha+beta, beta); split into items of at most
//    kM2lChunk terms, each item one accumulator of one beta.
//  m2m terms, grouped by alpha: (beta <= alpha, alpha - beta) with C(alpha, beta).
//  l2l terms, grouped by gamma: (beta >= gamma, beta - gamma) with C(beta, gamma).
constexpr int kM2lChunk = 8;
struct DerivEntry {
    int16_t e1[3], e2[3];
    int16_t k, pad;
};
struct TermEntry {        // one product coef * A[a] * B[b]
    uint8_t a, b;         // indices into the two operand arrays
    uint16_t pad;
    float coef32;
    double coef64;
};
struct ItemEntry {        // a run of terms with one output coefficient
    uint16_t out, first, len, pad;
};

struct Tables {
    int p, nt;
    int n_m2l_items, n_m2l_terms, n_shift_terms;
    short3* mi;                 // (a, b, c) per coefficient
    DerivEntry* deriv;
    ItemEntry* m2l_items;
    int* m2l_item_off;          // [nt + 1]: items of output coefficient beta (items are sorted by beta)
    TermEntry* m2l_terms;       // a = alpha (index into M), b = alpha + beta (index into T)
    int* m2m_off;               // [nt + 1] offsets into m2m_terms, by alpha
    TermEntry* m2m_terms;       // a = beta (index into child M), b = alpha - beta (monomial index)
    int* l2l_off;               // [nt + 1] by gamma
    TermEntry* l2l_terms;       // a = beta (index into parent L), b = beta - gamma (monomial index)
    double* mscale;             // [nt] (-1)^|alpha| / alpha!  (scaled multipoles of the M2L)
    double* lscale;             // [nt] 1 / beta!  (local coefficients from the scaled M2L sums)
};

}  // namespace fmm
}  // namespace gtap

namespace gtap {
namespace fmm {

// Device buffers of the tree build (owned by the plan).
struct TreeBufs {
    long long n;
    int leaf;
    const double* pos;            // input positions, n x 3 (device)
    const double* q;              // input charges (device)
    double* box;                  // [8]: lo x/y/z, side, scale
    double* bbox_part;            // [6 * kBoxParts]
    unsigned long long* keys[2];  // radix-sort ping-pong
    uint32_t* vals[2];
    int* hist;                    // [256 * ntiles]
    int* hist_scan;
    int* tile_sums;               // scan scratch
    Dbl4* geom;
    int4* info;
    int4* lat;                    // cell centre on the level-21 lattice: (2i+1) << (21 - level) per axis, level
    int cap_cells;
    int* lstart;                  // [kMaxLevel + 3]: first cell of each level
    int* lvl_n;                   // [kMaxLevel + 1]: cells per level
    int* lvl_total;               // [kMaxLevel + 1]: children created per level
    int* cnt;                     // [cap_cells] per-level child counts
    int* off;                     // [cap_cells] their exclusive scan
    int* bounds;                  // [9 * cap_cells] octant boundaries
    int* flags;                   // [4]: [0] cell capacity exceeded, [1] malformed record, [2] leaves, [3] largest leaf
    Dbl4* pts;                 // sorted points {x, y, z, q}
    float4* ploc;                 // sorted points relative to their leaf centre {x, y, z, q} (FP32)
    const uint32_t* order;        // sorted position -> input index (one of vals[])
    const unsigned long long* codes;   // sorted Morton codes (one of keys[])
};
constexpr int kBoxParts = 304;

int radix_tiles(long long n);
// Tree build in three stream-ordered parts: bounding box, Morton codes and
// radix sort; refinement of levels [l0, l1); then the start entries of levels
// left unrefined (all empty), the gather of points into tree order, and the
// structural check of the cell records (flags[1..3]).
cudaError_t launch_tree_sort(TreeBufs& b, cudaStream_t s);
cudaError_t launch_tree_levels(const TreeBufs& b, int l0, int l1, cudaStream_t s);
cudaError_t launch_tree_finish(const TreeBufs& b, int levels_done, cudaStream_t s);
// Leaf-local FP32 coordinates (needs the cell count, known after the build).
cudaError_t launch_leaf_local(const TreeBufs& b, int n_cells, cudaStream_t s);

// Evaluation (fmm_eval.cu).  R = float (mixed) or double.
struct EvalBufs {
    int p, nt, n_cells, n_levels;
    long long n;
    const Dbl4* geom;
    const int4* info;
    const int4* lat;              // lattice centres (see TreeBufs)
    float lat_unit;               // side / 2^22: length of one lattice step
    const int* lstart;            // host copy of the level starts
    const Dbl4* pts;
    const float4* ploc;
    const uint32_t* order;
    double* M;                    // [n_cells * nt]
    double* L;
    Tables tab;                   // device tables
    // lists grouped by target (CSR)
    const int* m2l_off;           // [n_cells + 1]
    const int* m2l_src;
    const int* p2p_off;
    const int* p2p_src;
    double* phi;                  // output, input order
    void* m2l_ms;                 // scaled multipoles for M2L (FP32 rows mixed, FP64 rows otherwise)
};
size_t m2l_scratch_bytes(int p, int n_cells, bool mixed);
cudaError_t launch_upward(const EvalBufs& e, bool mixed, int fp64_levels, cudaStream_t s);
cudaError_t launch_m2l(const EvalBufs& e, bool mixed, cudaStream_t s);
cudaError_t launch_downward(const EvalBufs& e, bool mixed, int fp64_levels, cudaStream_t s);
cudaError_t launch_leaf_eval(const EvalBufs& e, bool mixed, cudaStream_t s);
// Group list entries (target << 32 | source) by target: off[n_cells + 1], src[count].
cudaError_t launch_group(const unsigned long long* list, long long count, int n_cells, int* cnt, int* off,
                         int* cursor, int* src, int* tile_sums, cudaStream_t s);

// Environment of a traversal rooted at (target, source) of a built plan.
gtap_status dtt_env(const gtap_fmm* plan, int target, int source, DttEnv* out);

}  // namespace fmm
}  // namespace gtap
