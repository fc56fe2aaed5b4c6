// Data-parallel FMM kernels around the traversal (Sec. 6.4.1): upward pass
// (P2M at leaves, M2M level by level), M2L over the interaction list grouped
// by target cell, downward pass (L2L level by level) and the leaf kernel
// (L2P + P2P over the near-field list).  Cartesian Taylor expansions of total
// order p about the cell centres:
//   P2M  M_a  = sum_j q_j (x_j - c)^a
//   M2M  M_a(c) += sum_{b <= a} C(a, b) (c' - c)^(a-b) M_b(c')      (child c')
//   M2L  L_b(A) += sum_{|a|+|b| <= p} (-1)^|a| C(a+b, b) T_{a+b}(c_A - c_B) M_a(B)
//   L2L  L_g(c') += sum_{b >= g} C(b, g) (c' - c)^(b-g) L_b(c)       (child c')
//   L2P  phi_i += sum_b L_b (x_i - c)^b
//   P2P  phi_i += sum_{j != i} q_j / |x_i - x_j|
// with T_n = d^n(1/r)/n! from the recurrence in fmm_internal.h.  R is the
// arithmetic type: double, or float for the mixed form, where the per-target
// sums of M2L and P2P are compensated (Kahan) and the translations into the
// top levels stay in double.
#include <cuda_runtime.h>

#include <type_traits>

#include "fmm_internal.h"
#include "scan.cuh"

namespace gtap {
namespace fmm {
namespace {

template <class R> struct Ops;
template <> struct Ops<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double rsq(double a) { return rsqrt(a); }
    static __device__ __forceinline__ double coef(const TermEntry& t) { return t.coef64; }
};
template <> struct Ops<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float rsq(float a) { return rsqrtf(a); }
    static __device__ __forceinline__ float coef(const TermEntry& t) { return t.coef32; }
};

// Compensated accumulator (Kahan) for float; plain sum for double.
template <class R> struct Acc {
    R s = 0, c = 0;
    __device__ __forceinline__ void add(R v) {
        if constexpr (sizeof(R) == 4) {
            const R y = Ops<R>::sub(v, c);
            const R t = Ops<R>::add(s, y);
            c = Ops<R>::sub(Ops<R>::sub(t, s), y);
            s = t;
        } else {
            s += v;
        }
    }
};

// Index table (a, b, c) -> coefficient, (p+1)^3 shorts, in shared memory.
__device__ __forceinline__ void load_index(const Tables& tb, short* idx) {
    const int p1 = tb.p + 1;
    for (int i = threadIdx.x; i < p1 * p1 * p1; i += blockDim.x) idx[i] = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < tb.nt; i += blockDim.x) {
        const short3 m = tb.mi[i];
        idx[(m.x * p1 + m.y) * p1 + m.z] = (short)i;
    }
    __syncthreads();
}

// Monomials x^a y^b z^c of one displacement for every coefficient, by the
// nested powers (no table of powers needed).
template <class R>
__device__ __forceinline__ void monomials(int p, const short* idx, R x, R y, R z, R* out) {
    const int p1 = p + 1;
    R xa = 1;
    for (int a = 0; a <= p; ++a) {
        R xab = xa;
        for (int b = 0; a + b <= p; ++b) {
            R t = xab;
            for (int c = 0; a + b + c <= p; ++c) {
                out[idx[(a * p1 + b) * p1 + c]] = t;
                t = Ops<R>::mul(t, z);
            }
            xab = Ops<R>::mul(xab, y);
        }
        xa = Ops<R>::mul(xa, x);
    }
}

// ---------------------------------------------------------------------------
// P2M: one block per leaf.  Point powers in shared memory, one thread per
// coefficient summing over the leaf's points in order.
template <class R>
__global__ void k_p2m(EvalBufs e) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int p = e.p, nt = e.nt, p1 = p + 1;
    R* pw = reinterpret_cast<R*>(sm_raw);              // [kMaxLeaf][3][p1]
    R* qv = pw + kMaxLeaf * 3 * p1;                    // [kMaxLeaf]
    short3* mi = reinterpret_cast<short3*>(qv + kMaxLeaf);
    for (int i = threadIdx.x; i < nt; i += blockDim.x) mi[i] = e.tab.mi[i];
    for (int c = blockIdx.x; c < e.n_cells; c += gridDim.x) {
        const int4 in = e.info[c];
        if (in.z >= 0) continue;
        const Dbl4 g = e.geom[c];
        __syncthreads();
        for (int k = threadIdx.x; k < in.y; k += blockDim.x) {
            R d[3];
            if constexpr (sizeof(R) == 4) {
                const float4 pl = e.ploc[in.x + k];
                d[0] = pl.x; d[1] = pl.y; d[2] = pl.z;
                qv[k] = pl.w;
            } else {
                const Dbl4 pt = e.pts[in.x + k];
                d[0] = __dsub_rn(pt.x, g.x); d[1] = __dsub_rn(pt.y, g.y); d[2] = __dsub_rn(pt.z, g.z);
                qv[k] = pt.w;
            }
            for (int a = 0; a < 3; ++a) {
                R v = 1;
                pw[(k * 3 + a) * p1] = v;
                for (int j = 1; j <= p; ++j) { v = Ops<R>::mul(v, d[a]); pw[(k * 3 + a) * p1 + j] = v; }
            }
        }
        __syncthreads();
        for (int a = threadIdx.x; a < nt; a += blockDim.x) {
            const short3 m = mi[a];
            Acc<R> acc;
            for (int k = 0; k < in.y; ++k) {
                const R t = Ops<R>::mul(Ops<R>::mul(Ops<R>::mul(qv[k], pw[(k * 3) * p1 + m.x]), pw[(k * 3 + 1) * p1 + m.y]),
                                        pw[(k * 3 + 2) * p1 + m.z]);
                acc.add(t);
            }
            e.M[(size_t)c * nt + a] = (double)acc.s - (double)acc.c;
        }
    }
}

// M2M for the parents of one level: one block per parent.
template <class R>
__global__ void k_m2m(EvalBufs e, int lo, int hi) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int p = e.p, nt = e.nt, p1 = p + 1;
    R* mono = reinterpret_cast<R*>(sm_raw);            // [8][nt]
    R* mc = mono + 8 * nt;                             // [8][nt]
    short* idx = reinterpret_cast<short*>(mc + 8 * nt);
    load_index(e.tab, idx);
    for (int c = lo + blockIdx.x; c < hi; c += gridDim.x) {
        const int4 in = e.info[c];
        if (in.z < 0) continue;
        const int nch = in.w & 0xFF, cf = in.z;
        const Dbl4 g = e.geom[c];
        __syncthreads();
        if ((int)threadIdx.x < nch) {
            const Dbl4 gc = e.geom[cf + threadIdx.x];
            monomials<R>(p, idx, (R)__dsub_rn(gc.x, g.x), (R)__dsub_rn(gc.y, g.y), (R)__dsub_rn(gc.z, g.z),
                         mono + threadIdx.x * nt);
        }
        for (int i = threadIdx.x; i < nch * nt; i += blockDim.x) mc[i] = (R)e.M[(size_t)cf * nt + i];
        __syncthreads();
        for (int a = threadIdx.x; a < nt; a += blockDim.x) {
            const int t0 = e.tab.m2m_off[a], t1 = e.tab.m2m_off[a + 1];
            Acc<R> acc;
            for (int j = 0; j < nch; ++j) {
                R s = 0;
                for (int t = t0; t < t1; ++t) {
                    const TermEntry te = e.tab.m2m_terms[t];
                    s += Ops<R>::coef(te) * mono[j * nt + te.b] * mc[j * nt + te.a];
                }
                acc.add(s);
            }
            e.M[(size_t)c * nt + a] = (double)acc.s - (double)acc.c;
        }
    }
    (void)p1;
}

// ---------------------------------------------------------------------------
// M2L: one block per target cell; sources in batches of kSB.  The Taylor
// coefficients of every source displacement are built degree by degree in
// shared memory, then each thread owns one item (a run of <= kM2lChunk terms
// of one output coefficient) and accumulates it over all sources.
constexpr int kSB = 8;

template <class R>
__global__ void k_m2l(EvalBufs e) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int p = e.p, nt = e.nt;
    R* T = reinterpret_cast<R*>(sm_raw);               // [kSB][nt]
    R* Ms = T + kSB * nt;                              // [kSB][nt]
    R* dv = Ms + kSB * nt;                             // [kSB][4]: dx, dy, dz, 1/r^2
    R* accs = dv + kSB * 4;                            // [n_items]
    R* c1 = accs + e.tab.n_m2l_items;                  // [p + 1]
    R* c2 = c1 + (p + 1);
    DerivEntry* der = reinterpret_cast<DerivEntry*>(c2 + (p + 1) + ((p + 1) & 1) + 2);
    for (int i = threadIdx.x; i < nt; i += blockDim.x) der[i] = e.tab.deriv[i];
    for (int k = threadIdx.x; k <= p; k += blockDim.x) {
        c1[k] = k ? (R)(2.0 * k - 1.0) / (R)k : (R)0;
        c2[k] = k ? (R)(k - 1.0) / (R)k : (R)0;
    }
    // this thread's item, its terms cached in registers
    const int it = threadIdx.x;
    const bool has_item = it < e.tab.n_m2l_items;
    int len = 0;
    R cf[kM2lChunk];
    uint8_t ta[kM2lChunk], tb[kM2lChunk];
    if (has_item) {
        const ItemEntry ie = e.tab.m2l_items[it];
        len = ie.len;
#pragma unroll
        for (int j = 0; j < kM2lChunk; ++j) {
            if (j < len) {
                const TermEntry te = e.tab.m2l_terms[ie.first + j];
                cf[j] = Ops<R>::coef(te);
                ta[j] = te.a;
                tb[j] = te.b;
            } else {
                cf[j] = 0; ta[j] = 0; tb[j] = 0;
            }
        }
    }
    for (int c = blockIdx.x; c < e.n_cells; c += gridDim.x) {
        const int s0 = e.m2l_off[c], s1 = e.m2l_off[c + 1];
        if (s0 == s1) continue;
        const Dbl4 g = e.geom[c];
        Acc<R> acc;
        for (int b0 = s0; b0 < s1; b0 += kSB) {
            const int nb = min(kSB, s1 - b0);
            __syncthreads();
            for (int i = threadIdx.x; i < nb * nt; i += blockDim.x) {
                const int s = i / nt, a = i - s * nt;
                Ms[i] = (R)e.M[(size_t)e.m2l_src[b0 + s] * nt + a];
            }
            if ((int)threadIdx.x < nb) {
                const Dbl4 gs = e.geom[e.m2l_src[b0 + threadIdx.x]];
                const R x = (R)__dsub_rn(g.x, gs.x), y = (R)__dsub_rn(g.y, gs.y), z = (R)__dsub_rn(g.z, gs.z);
                const R r2 = x * x + y * y + z * z;
                R* d = dv + threadIdx.x * 4;
                d[0] = x; d[1] = y; d[2] = z; d[3] = (R)1 / r2;
                T[threadIdx.x * nt] = Ops<R>::rsq(r2);
            }
            __syncthreads();
            for (int k = 1; k <= p; ++k) {
                const int i0 = n_coef(k - 1), cnt = n_coef(k) - i0;
                for (int w = threadIdx.x; w < nb * cnt; w += blockDim.x) {
                    const int s = w / cnt, i = i0 + (w - s * cnt);
                    const DerivEntry de = der[i];
                    const R* Ts = T + s * nt;
                    const R* d = dv + s * 4;
                    R s1v = 0, s2v = 0;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if (de.e1[q] >= 0) s1v += d[q] * Ts[de.e1[q]];
                        if (de.e2[q] >= 0) s2v += Ts[de.e2[q]];
                    }
                    T[s * nt + i] = -(c1[k] * s1v + c2[k] * s2v) * d[3];
                }
                __syncthreads();
            }
            if (has_item) {
                for (int s = 0; s < nb; ++s) {
                    R part = 0;
#pragma unroll
                    for (int j = 0; j < kM2lChunk; ++j)
                        if (j < len) part += cf[j] * T[s * nt + tb[j]] * Ms[s * nt + ta[j]];
                    acc.add(part);
                }
            }
        }
        if (has_item) accs[it] = Ops<R>::sub(acc.s, acc.c);
        __syncthreads();
        for (int b = threadIdx.x; b < nt; b += blockDim.x) {
            Acc<R> sum;
            for (int i = e.tab.m2l_item_off[b]; i < e.tab.m2l_item_off[b + 1]; ++i) sum.add(accs[i]);
            e.L[(size_t)c * nt + b] = (double)sum.s - (double)sum.c;
        }
    }
}

// M2L in FP32 with the whole expansion in registers, one warp per target
// cell and one source cell per lane.  In the scaled variables
//   Tt_n = n! T_n,   Mt_a = (-1)^|a| M_a / a!,   Lt_b = b! L_b
// the translation is a plain correlation, Lt_b = sum_a Tt_{a+b} Mt_a, one FMA
// per term, and the recurrence for Tt has compile-time coefficients:
//   |n| r^2 Tt_n = -(2|n|-1) sum_i n_i x_i Tt_{n-e_i} - (|n|-1) sum_i n_i (n_i-1) Tt_{n-2e_i}.
// The order P is a template parameter so that every index is a constant and
// the compiler keeps Tt and Lt in registers.
__host__ __device__ constexpr int cidx(int a, int b, int c) {
    return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}
__host__ __device__ constexpr int row_stride(int p) { return (n_coef(p) + 3) / 4 * 4; }

template <int P>
__device__ __forceinline__ void taylor_scaled(float x, float y, float z, float* T) {
    const float r2 = x * x + y * y + z * z;
    const float ir = rsqrtf(r2);
    const float ir2 = ir * ir;
    T[0] = ir;
#pragma unroll
    for (int k = 1; k <= P; ++k) {
        const float ck = -(2.f * k - 1.f) / (float)k, dk = -((float)k - 1.f) / (float)k;
#pragma unroll
        for (int a = k; a >= 0; --a) {
#pragma unroll
            for (int b = k - a; b >= 0; --b) {
                const int c = k - a - b;
                float acc = 0.f;
                if (a > 0) acc += (ck * a) * x * T[cidx(a - 1, b, c)];
                if (b > 0) acc += (ck * b) * y * T[cidx(a, b - 1, c)];
                if (c > 0) acc += (ck * c) * z * T[cidx(a, b, c - 1)];
                if (a > 1) acc += (dk * a * (a - 1)) * T[cidx(a - 2, b, c)];
                if (b > 1) acc += (dk * b * (b - 1)) * T[cidx(a, b - 2, c)];
                if (c > 1) acc += (dk * c * (c - 1)) * T[cidx(a, b, c - 2)];
                T[cidx(a, b, c)] = acc * ir2;
            }
        }
    }
}

// Ms[cell][row_stride(P)] = (-1)^|a| M_a / a! in FP32; the factors come from a
// per-coefficient table (an FP64 divide is a long sequence on the FP64 pipe,
// the narrowest pipe of this GPU).
template <int P>
__global__ void k_scale_m(const double* __restrict__ M, int n_cells, const double* __restrict__ mscale,
                          float* __restrict__ Ms) {
    constexpr int N = n_coef(P), S = row_stride(P);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n_cells * S;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / S), j = (int)(i - (long long)c * S);
        Ms[i] = (j < N) ? (float)(M[(size_t)c * N + j] * __ldg(mscale + j)) : 0.f;
    }
}

// 3 resident blocks per SM (at most 168 registers, a few spills) measured 5 % faster than
// the unconstrained 229 registers at 2 blocks, and than 4 blocks with heavy spilling.
template <int P>
__global__ void __launch_bounds__(128, 3) k_m2l_reg(EvalBufs e, const float* __restrict__ Ms) {
    constexpr int N = n_coef(P), S = row_stride(P);
    const int lane = threadIdx.x & 31;
    const int tgt = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (tgt >= e.n_cells) return;
    const int s0 = e.m2l_off[tgt], s1 = e.m2l_off[tgt + 1];
    if (s0 == s1) return;
    // exact integer displacement on the level-21 lattice, one FP32 scaling
    const int4 lt = e.lat[tgt];
    const float u = e.lat_unit;
    float L[N];
#pragma unroll
    for (int i = 0; i < N; ++i) L[i] = 0.f;
    for (int base = s0; base < s1; base += 32) {
        const int s = base + lane;
        const bool valid = s < s1;
        const int src = valid ? e.m2l_src[s] : e.m2l_src[s0];
        const int4 ls = __ldg(e.lat + src);
        const float x = (float)(lt.x - ls.x) * u, y = (float)(lt.y - ls.y) * u, z = (float)(lt.z - ls.z) * u;
        float T[N];
        taylor_scaled<P>(x, y, z, T);
        const float wgt = valid ? 1.f : 0.f;
        const float4* row = reinterpret_cast<const float4*>(Ms + (size_t)src * S);
        float4 mv = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k1 = 0; k1 <= P; ++k1)
#pragma unroll
            for (int a1 = k1; a1 >= 0; --a1)
#pragma unroll
                for (int b1 = k1 - a1; b1 >= 0; --b1) {
                    const int c1 = k1 - a1 - b1;
                    const int ia = cidx(a1, b1, c1);
                    if ((ia & 3) == 0) mv = __ldg(row + ia / 4);
                    const float m = wgt * ((ia & 3) == 0 ? mv.x : (ia & 3) == 1 ? mv.y : (ia & 3) == 2 ? mv.z : mv.w);
#pragma unroll
                    for (int k2 = 0; k2 <= P - k1; ++k2)
#pragma unroll
                        for (int a2 = k2; a2 >= 0; --a2)
#pragma unroll
                            for (int b2 = k2 - a2; b2 >= 0; --b2) {
                                const int c2 = k2 - a2 - b2;
                                L[cidx(a2, b2, c2)] = fmaf(T[cidx(a1 + a2, b1 + b2, c1 + c2)], m, L[cidx(a2, b2, c2)]);
                            }
                }
    }
    // sum the lanes' partial expansions, then lane l writes L_b = Lt_b / b! for
    // b = l, l + 32, l + 64 (selected by register moves; one FP64 multiply each)
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float v = L[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        L[i] = v;
    }
    constexpr int R = (N + 31) / 32;
    float w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if ((i & 31) == lane) w[i >> 5] = L[i];
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (lane + 32 * r < N) e.L[(size_t)tgt * N + lane + 32 * r] = (double)w[r] * __ldg(e.tab.lscale + lane + 32 * r);
}

// FP64 M2L in the same scaled form: the local expansion stays in registers,
// the Taylor coefficients of each lane's source go to the lane's column of a
// shared-memory table (FP64 registers cannot hold both).  The FP64 pipe, not
// the shared-memory bandwidth, bounds this kernel.
template <int P>
__global__ void k_scale_m64(const double* __restrict__ M, int n_cells, const double* __restrict__ mscale,
                            double* __restrict__ Ms) {
    constexpr int N = n_coef(P), S = row_stride(P);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n_cells * S;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / S), j = (int)(i - (long long)c * S);
        Ms[i] = (j < N) ? M[(size_t)c * N + j] * __ldg(mscale + j) : 0.0;
    }
}

constexpr int kM2l64Warps = 4;

template <int P>
__global__ void __launch_bounds__(32 * kM2l64Warps) k_m2l_reg64(EvalBufs e, const double* __restrict__ Ms) {
    constexpr int N = n_coef(P), S = row_stride(P);
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double* T = reinterpret_cast<double*>(sm_raw) + (size_t)wib * N * 32 + lane;   // T[i * 32]
    const int tgt = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (tgt >= e.n_cells) return;
    const int s0 = e.m2l_off[tgt], s1 = e.m2l_off[tgt + 1];
    if (s0 == s1) return;
    const Dbl4 g = e.geom[tgt];
    double L[N];
#pragma unroll
    for (int i = 0; i < N; ++i) L[i] = 0.0;
    for (int base = s0; base < s1; base += 32) {
        const int s = base + lane;
        const bool valid = s < s1;
        const int src = valid ? e.m2l_src[s] : e.m2l_src[s0];
        const Dbl4 gs = e.geom[src];
        const double x = __dsub_rn(g.x, gs.x), y = __dsub_rn(g.y, gs.y), z = __dsub_rn(g.z, gs.z);
        const double r2 = x * x + y * y + z * z;
        const double ir2 = 1.0 / r2;
        T[0] = rsqrt(r2);
#pragma unroll
        for (int k = 1; k <= P; ++k) {
            const double ck = -(2.0 * k - 1.0) / (double)k, dk = -((double)k - 1.0) / (double)k;
#pragma unroll
            for (int a = k; a >= 0; --a)
#pragma unroll
                for (int b = k - a; b >= 0; --b) {
                    const int c = k - a - b;
                    double acc = 0.0;
                    if (a > 0) acc += (ck * a) * x * T[32 * cidx(a - 1, b, c)];
                    if (b > 0) acc += (ck * b) * y * T[32 * cidx(a, b - 1, c)];
                    if (c > 0) acc += (ck * c) * z * T[32 * cidx(a, b, c - 1)];
                    if (a > 1) acc += (dk * a * (a - 1)) * T[32 * cidx(a - 2, b, c)];
                    if (b > 1) acc += (dk * b * (b - 1)) * T[32 * cidx(a, b - 2, c)];
                    if (c > 1) acc += (dk * c * (c - 1)) * T[32 * cidx(a, b, c - 2)];
                    T[32 * cidx(a, b, c)] = acc * ir2;
                }
        }
        const double wgt = valid ? 1.0 : 0.0;
        const double2* row = reinterpret_cast<const double2*>(Ms + (size_t)src * S);
        double2 mv = make_double2(0.0, 0.0);
#pragma unroll
        for (int k1 = 0; k1 <= P; ++k1)
#pragma unroll
            for (int a1 = k1; a1 >= 0; --a1)
#pragma unroll
                for (int b1 = k1 - a1; b1 >= 0; --b1) {
                    const int c1 = k1 - a1 - b1;
                    const int ia = cidx(a1, b1, c1);
                    if ((ia & 1) == 0) mv = __ldg(row + ia / 2);
                    const double m = wgt * ((ia & 1) == 0 ? mv.x : mv.y);
#pragma unroll
                    for (int k2 = 0; k2 <= P - k1; ++k2)
#pragma unroll
                        for (int a2 = k2; a2 >= 0; --a2)
#pragma unroll
                            for (int b2 = k2 - a2; b2 >= 0; --b2) {
                                const int c2 = k2 - a2 - b2;
                                L[cidx(a2, b2, c2)] = fma(T[32 * cidx(a1 + a2, b1 + b2, c1 + c2)], m, L[cidx(a2, b2, c2)]);
                            }
                }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double v = L[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        L[i] = v;
    }
    constexpr int R = (N + 31) / 32;
    double w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if ((i & 31) == lane) w[i >> 5] = L[i];
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (lane + 32 * r < N) e.L[(size_t)tgt * N + lane + 32 * r] = w[r] * __ldg(e.tab.lscale + lane + 32 * r);
}

// L2L from the parents of one level into their children: one block per parent.
template <class R>
__global__ void k_l2l(EvalBufs e, int lo, int hi) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int p = e.p, nt = e.nt;
    R* mono = reinterpret_cast<R*>(sm_raw);            // [8][nt]
    R* lp = mono + 8 * nt;                             // [nt]
    short* idx = reinterpret_cast<short*>(lp + nt);
    load_index(e.tab, idx);
    for (int c = lo + blockIdx.x; c < hi; c += gridDim.x) {
        const int4 in = e.info[c];
        if (in.z < 0) continue;
        const int nch = in.w & 0xFF, cf = in.z;
        const Dbl4 g = e.geom[c];
        __syncthreads();
        if ((int)threadIdx.x < nch) {
            const Dbl4 gc = e.geom[cf + threadIdx.x];
            monomials<R>(p, idx, (R)__dsub_rn(gc.x, g.x), (R)__dsub_rn(gc.y, g.y), (R)__dsub_rn(gc.z, g.z),
                         mono + threadIdx.x * nt);
        }
        for (int i = threadIdx.x; i < nt; i += blockDim.x) lp[i] = (R)e.L[(size_t)c * nt + i];
        __syncthreads();
        for (int w = threadIdx.x; w < nch * nt; w += blockDim.x) {
            const int j = w / nt, gi = w - j * nt;
            const int t0 = e.tab.l2l_off[gi], t1 = e.tab.l2l_off[gi + 1];
            R s = 0;
            for (int t = t0; t < t1; ++t) {
                const TermEntry te = e.tab.l2l_terms[t];
                s += Ops<R>::coef(te) * mono[j * nt + te.b] * lp[te.a];
            }
            e.L[(size_t)(cf + j) * nt + gi] += (double)s;
        }
    }
}

// Packed FP32 pairs (two lanes of a 64-bit register) for the P2P inner loop:
// one f32x2 instruction does the work of two FP32 ones.
__device__ __forceinline__ unsigned long long pack_f32x2(float lo, float hi) {
    return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float lo_f32(unsigned long long v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float hi_f32(unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ unsigned long long sub_f32x2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long mul_f32x2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// 1/sqrt(x), the hardware approximation (inputs here are normal: distinct points)
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// Leaf kernel: one block per leaf.  Threads are (target slot, source part):
// each thread sums over every parts-th source point of the near-field list,
// source points staged in shared memory in batches of up to kSrcBatch from
// consecutive source leaves; then the parts are combined and L2P added.
constexpr int kLeafBlock = 128;
constexpr int kSrcBatch = 1024;

template <class R>
__global__ void __launch_bounds__(kLeafBlock) k_leaf(EvalBufs e) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int p = e.p, nt = e.nt;
    using R4 = typename std::conditional<sizeof(R) == 4, float4, Dbl4>::type;
    R4* sp = reinterpret_cast<R4*>(sm_raw);             // [kSrcBatch] source x, y, z, q
    int* sid = reinterpret_cast<int*>(sp + kSrcBatch);  // [kSrcBatch] sorted index
    R* red = reinterpret_cast<R*>(sid + kSrcBatch);     // [kLeafBlock] (and a compensation array)
    R* redc = red + kLeafBlock;
    R* lsm = redc + kLeafBlock;                         // [nt]
    int* bpre = reinterpret_cast<int*>(lsm + nt + (nt & 1));  // [33] prefix of the batch's source counts
    int* bfirst = bpre + 34;                            // [32]
    R* boff = reinterpret_cast<R*>(bfirst + 32);        // [32][3] source-centre offsets (mixed)
    int* bnum = reinterpret_cast<int*>(boff + 96);      // [1]
    short* idx = reinterpret_cast<short*>(bnum + 4);
    load_index(e.tab, idx);
    const int t = threadIdx.x, lane = t & 31;
    for (int c = blockIdx.x; c < e.n_cells; c += gridDim.x) {
        const int4 in = e.info[c];
        if (in.z >= 0) continue;
        const Dbl4 g = e.geom[c];
        // one slot per target point, kLeafBlock / count source parts per slot
        const int count = in.y;
        const int tp = max(count, 1);
        const int parts = kLeafBlock / tp;
        const int part = t / tp, slot = t - part * tp;
        const bool active = part < parts;
        const int ki = in.x + (active ? slot : 0);
        R xi, yi, zi;
        if constexpr (sizeof(R) == 4) {
            const float4 pl = e.ploc[ki];
            xi = pl.x; yi = pl.y; zi = pl.z;
        } else {
            const Dbl4 pt = e.pts[ki];
            xi = pt.x; yi = pt.y; zi = pt.z;
        }
        __syncthreads();
        for (int i = t; i < nt; i += kLeafBlock) lsm[i] = (R)e.L[(size_t)c * nt + i];
        Acc<R> acc;
        if constexpr (sizeof(R) == 4) {
            // the leaf's own points first: the target's own copy has exactly the same
            // local coordinates (r^2 == 0) and is the only source that can, so only this
            // pass tests for it; the batches below skip the leaf itself
            __syncthreads();
            for (int i = t; i < count; i += kLeafBlock) sp[i] = e.ploc[in.x + i];
            __syncthreads();
            if (active) {
                float bsum = 0.f;
                for (int j = part; j < count; j += parts) {
                    const float4 sj = sp[j];
                    const float dx = xi - sj.x, dy = yi - sj.y, dz = zi - sj.z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    bsum += (r2 > 0.f) ? sj.w * rsqrtf(r2) : 0.f;
                }
                acc.add(bsum);
            }
        }
        const int s0 = e.p2p_off[c], s1 = e.p2p_off[c + 1];
        int cur = s0;
        while (cur < s1) {
            __syncthreads();
            if (t < 32) {
                const int j = cur + lane;
                int cnt = 0, first = 0;
                Dbl4 gs = make_dbl4(0, 0, 0, 0);
                if (j < s1) {
                    const int sc = e.p2p_src[j];
                    const int4 si = e.info[sc];
                    cnt = (sizeof(R) == 4 && sc == c) ? 0 : si.y;   // FP32: the own leaf had its pass
                    first = si.x;
                    gs = e.geom[sc];
                }
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const unsigned fit = __ballot_sync(0xffffffffu, j < s1 && incl <= kSrcBatch);
                const int nfit = max(1, __popc(fit));   // fit is a prefix of lanes; a leaf holds <= 64 points
                if (lane < nfit) {
                    bpre[lane + 1] = incl;
                    bfirst[lane] = first;
                    if constexpr (sizeof(R) == 4) {
                        boff[lane * 3 + 0] = (R)__dsub_rn(gs.x, g.x);
                        boff[lane * 3 + 1] = (R)__dsub_rn(gs.y, g.y);
                        boff[lane * 3 + 2] = (R)__dsub_rn(gs.z, g.z);
                    }
                }
                if (lane == 0) { bpre[0] = 0; bnum[0] = nfit; }
            }
            __syncthreads();
            const int nfit = bnum[0];
            const int total = bpre[nfit];
            if constexpr (sizeof(R) == 4) {
                // pair records {x0 x1 | y0 y1 | z0 z1 | q0 q1} of source points 2m, 2m+1
                // (an odd tail is padded with a far, chargeless point)
                float4* pr = reinterpret_cast<float4*>(sp);
                for (int m = t; 2 * m < total; m += kLeafBlock) {
                    const int i0 = 2 * m;
                    int a = 0, b = nfit - 1;   // last source leaf with bpre[s] <= i0
                    while (a < b) {
                        const int mid = (a + b + 1) >> 1;
                        if (bpre[mid] <= i0) a = mid; else b = mid - 1;
                    }
                    const float4 l0 = e.ploc[bfirst[a] + (i0 - bpre[a])];
                    const float4 p0 = make_float4(l0.x + boff[a * 3], l0.y + boff[a * 3 + 1], l0.z + boff[a * 3 + 2], l0.w);
                    float4 p1 = make_float4(1e18f, 1e18f, 1e18f, 0.f);
                    if (i0 + 1 < total) {
                        int a1 = a;   // skips empty entries (the target's own leaf counts 0 here)
                        while (a1 + 1 < nfit && bpre[a1 + 1] <= i0 + 1) ++a1;
                        const float4 l1 = e.ploc[bfirst[a1] + (i0 + 1 - bpre[a1])];
                        p1 = make_float4(l1.x + boff[a1 * 3], l1.y + boff[a1 * 3 + 1], l1.z + boff[a1 * 3 + 2], l1.w);
                    }
                    pr[2 * m] = make_float4(p0.x, p1.x, p0.y, p1.y);
                    pr[2 * m + 1] = make_float4(p0.z, p1.z, p0.w, p1.w);
                }
            } else {
                for (int i = t; i < total; i += kLeafBlock) {
                    int a = 0, b = nfit - 1;   // last source leaf with bpre[s] <= i
                    while (a < b) {
                        const int mid = (a + b + 1) >> 1;
                        if (bpre[mid] <= i) a = mid; else b = mid - 1;
                    }
                    const int k = bfirst[a] + (i - bpre[a]);
                    sid[i] = k;
                    sp[i] = e.pts[k];
                }
            }
            __syncthreads();
            if (active) {
                if constexpr (sizeof(R) == 4) {
                    // other leaves only: no self term.  Two source points per step in
                    // packed FP32 pairs; each batch is summed plainly and added to the
                    // compensated total
                    const unsigned long long X2 = pack_f32x2(xi, xi), Y2 = pack_f32x2(yi, yi), Z2 = pack_f32x2(zi, zi);
                    const ulonglong2* pr = reinterpret_cast<const ulonglong2*>(sp);
                    const int npairs = (total + 1) >> 1;
                    unsigned long long acc2 = 0ull;
#pragma unroll 2
                    for (int m = part; m < npairs; m += parts) {
                        const ulonglong2 xy = pr[2 * m], zq = pr[2 * m + 1];
                        const unsigned long long dx = sub_f32x2(X2, xy.x), dy = sub_f32x2(Y2, xy.y), dz = sub_f32x2(Z2, zq.x);
                        unsigned long long r2 = mul_f32x2(dx, dx);
                        r2 = fma_f32x2(dy, dy, r2);
                        r2 = fma_f32x2(dz, dz, r2);
                        const unsigned long long ir = pack_f32x2(rsqrt_ftz(lo_f32(r2)), rsqrt_ftz(hi_f32(r2)));
                        acc2 = fma_f32x2(zq.y, ir, acc2);
                    }
                    acc.add(lo_f32(acc2) + hi_f32(acc2));
                } else {
                    for (int j = part; j < total; j += parts) {
                        if (sid[j] == ki) continue;
                        const R4 s = sp[j];
                        const R dx = xi - s.x, dy = yi - s.y, dz = zi - s.z;
                        const R r2 = dx * dx + dy * dy + dz * dz;
                        acc.add(s.w * Ops<R>::rsq(r2));
                    }
                }
            }
            cur += nfit;
        }
        red[t] = acc.s;
        redc[t] = acc.c;
        __syncthreads();
        if (part == 0 && active) {
            Acc<R> tot;
            tot.s = red[t];
            tot.c = redc[t];
            for (int q = 1; q < parts; ++q) tot.add(Ops<R>::sub(red[q * tp + slot], redc[q * tp + slot]));
            // L2P
            R pl = 0;
            const int p1 = p + 1;
            R xa = 1;
            const R dx = (sizeof(R) == 4) ? xi : (R)__dsub_rn((double)xi, g.x);
            const R dy = (sizeof(R) == 4) ? yi : (R)__dsub_rn((double)yi, g.y);
            const R dz = (sizeof(R) == 4) ? zi : (R)__dsub_rn((double)zi, g.z);
            for (int a = 0; a <= p; ++a) {
                R xab = xa;
                for (int b = 0; a + b <= p; ++b) {
                    R m = xab;
                    for (int cc = 0; a + b + cc <= p; ++cc) {
                        pl += lsm[idx[(a * p1 + b) * p1 + cc]] * m;
                        m *= dz;
                    }
                    xab *= dy;
                }
                xa *= dx;
            }
            e.phi[e.order[ki]] = (double)tot.s - (double)tot.c + (double)pl;
        }
    }
}

// ---------------------------------------------------------------------------
// Counting sort of a list by target.  The traversal appends the child pairs of
// one split pair together, so a warp's 32 entries often share a target: the
// lanes of one target (found with __match_any_sync) make one atomic between
// them.  The warp-uniform loop keeps all 32 lanes in every collective.
__global__ void k_group_count(const unsigned long long* list, long long count, int* cnt) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); w < count; w += stride) {
        const long long i = w + lane;
        const int tg = (i < count) ? (int)(list[i] >> 32) : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, tg);
        if (tg >= 0 && lane == __ffs(grp) - 1) atomicAdd(&cnt[tg], __popc(grp));
    }
}

__global__ void k_group_fill(const unsigned long long* list, long long count, const int* off, int* cursor, int* src) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); w < count; w += stride) {
        const long long i = w + lane;
        const unsigned long long v = (i < count) ? list[i] : 0ull;
        const int tg = (i < count) ? (int)(v >> 32) : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, tg);
        const int leader = __ffs(grp) - 1;
        int base = 0;
        if (tg >= 0 && lane == leader) base = atomicAdd(&cursor[tg], __popc(grp));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (tg >= 0) src[off[tg] + base + __popc(grp & ((1u << lane) - 1u))] = (int)(v & 0xFFFFFFFFull);
    }
}

int grid_for(long long n, int block, int cap) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <class R>
size_t p2m_smem(int p, int nt) { return sizeof(R) * (kMaxLeaf * 3 * (p + 1) + kMaxLeaf) + sizeof(short3) * nt + 16; }
template <class R>
size_t m2m_smem(int p, int nt) { return sizeof(R) * 16 * nt + sizeof(short) * (p + 1) * (p + 1) * (p + 1) + 16; }
template <class R>
size_t l2l_smem(int p, int nt) { return sizeof(R) * 9 * nt + sizeof(short) * (p + 1) * (p + 1) * (p + 1) + 16; }
template <class R>
size_t m2l_smem(int p, int nt, int items) {
    return sizeof(R) * (2 * kSB * nt + 4 * kSB + items + 2 * (p + 1) + ((p + 1) & 1) + 2) + sizeof(DerivEntry) * nt + 16;
}
template <class R>
size_t leaf_smem(int p, int nt) {
    const size_t r4 = (sizeof(R) == 4) ? sizeof(float4) : sizeof(Dbl4);
    return r4 * kSrcBatch + sizeof(int) * kSrcBatch + sizeof(R) * (2 * kLeafBlock + nt + (nt & 1)) + sizeof(int) * 66 +
           sizeof(R) * 96 + sizeof(int) * 4 + sizeof(short) * (p + 1) * (p + 1) * (p + 1) + 16;
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class R>
cudaError_t upward_level(const EvalBufs& e, int l, cudaStream_t s) {
    const int lo = e.lstart[l], hi = e.lstart[l + 1];
    if (hi <= lo) return cudaSuccess;
    const size_t sm = m2m_smem<R>(e.p, e.nt);
    cudaError_t err = set_smem(k_m2m<R>, sm);
    if (err != cudaSuccess) return err;
    k_m2m<R><<<grid_for(hi - lo, 1, 1 << 20), 128, sm, s>>>(e, lo, hi);
    return cudaGetLastError();
}

template <class R>
cudaError_t downward_level(const EvalBufs& e, int l, cudaStream_t s) {
    const int lo = e.lstart[l], hi = e.lstart[l + 1];
    if (hi <= lo) return cudaSuccess;
    const size_t sm = l2l_smem<R>(e.p, e.nt);
    cudaError_t err = set_smem(k_l2l<R>, sm);
    if (err != cudaSuccess) return err;
    k_l2l<R><<<grid_for(hi - lo, 1, 1 << 20), 128, sm, s>>>(e, lo, hi);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_upward(const EvalBufs& e, bool mixed, int fp64_levels, cudaStream_t s) {
    cudaError_t err;
    const int grid = grid_for(e.n_cells, 1, 1 << 20);
    if (mixed) {
        const size_t sm = p2m_smem<float>(e.p, e.nt);
        if ((err = set_smem(k_p2m<float>, sm)) != cudaSuccess) return err;
        k_p2m<float><<<grid, 128, sm, s>>>(e);
    } else {
        const size_t sm = p2m_smem<double>(e.p, e.nt);
        if ((err = set_smem(k_p2m<double>, sm)) != cudaSuccess) return err;
        k_p2m<double><<<grid, 128, sm, s>>>(e);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    for (int l = e.n_levels - 2; l >= 0; --l) {
        err = (!mixed || l < fp64_levels) ? upward_level<double>(e, l, s) : upward_level<float>(e, l, s);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

template <int P>
cudaError_t launch_m2l_reg(const EvalBufs& e, float* ms, cudaStream_t s) {
    k_scale_m<P><<<grid_for((long long)e.n_cells * row_stride(P), 256, 4096), 256, 0, s>>>(e.M, e.n_cells, e.tab.mscale, ms);
    k_m2l_reg<P><<<grid_for((long long)e.n_cells * 32, 128, 1 << 30), 128, 0, s>>>(e, ms);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_m2l_reg64(const EvalBufs& e, double* ms, cudaStream_t s) {
    k_scale_m64<P><<<grid_for((long long)e.n_cells * row_stride(P), 256, 4096), 256, 0, s>>>(e.M, e.n_cells, e.tab.mscale, ms);
    const size_t sm = sizeof(double) * n_coef(P) * 32 * kM2l64Warps;
    cudaError_t err = set_smem(k_m2l_reg64<P>, sm);
    if (err != cudaSuccess) return err;
    k_m2l_reg64<P><<<grid_for((long long)e.n_cells * 32, 32 * kM2l64Warps, 1 << 30), 32 * kM2l64Warps, sm, s>>>(e, ms);
    return cudaGetLastError();
}

// Scratch for the scaled multipoles: FP32 rows (mixed) or FP64 rows, in bytes.
size_t m2l_scratch_bytes(int p, int n_cells, bool mixed) {
    return (size_t)n_cells * row_stride(p) * (mixed ? sizeof(float) : sizeof(double));
}

cudaError_t launch_m2l(const EvalBufs& e, bool mixed, cudaStream_t s) {
    cudaError_t err;
    if (e.m2l_ms != nullptr && e.p <= 6) {
        float* f32 = static_cast<float*>(e.m2l_ms);
        double* f64 = static_cast<double*>(e.m2l_ms);
        switch (e.p) {
        case 1: return mixed ? launch_m2l_reg<1>(e, f32, s) : launch_m2l_reg64<1>(e, f64, s);
        case 2: return mixed ? launch_m2l_reg<2>(e, f32, s) : launch_m2l_reg64<2>(e, f64, s);
        case 3: return mixed ? launch_m2l_reg<3>(e, f32, s) : launch_m2l_reg64<3>(e, f64, s);
        case 4: return mixed ? launch_m2l_reg<4>(e, f32, s) : launch_m2l_reg64<4>(e, f64, s);
        case 5: return mixed ? launch_m2l_reg<5>(e, f32, s) : launch_m2l_reg64<5>(e, f64, s);
        default: return mixed ? launch_m2l_reg<6>(e, f32, s) : launch_m2l_reg64<6>(e, f64, s);
        }
    }
    const int grid = grid_for(e.n_cells, 1, 1 << 20);
    const int block = (e.tab.n_m2l_items + 31) / 32 * 32;
    if (mixed) {
        const size_t sm = m2l_smem<float>(e.p, e.nt, e.tab.n_m2l_items);
        if ((err = set_smem(k_m2l<float>, sm)) != cudaSuccess) return err;
        k_m2l<float><<<grid, block, sm, s>>>(e);
    } else {
        const size_t sm = m2l_smem<double>(e.p, e.nt, e.tab.n_m2l_items);
        if ((err = set_smem(k_m2l<double>, sm)) != cudaSuccess) return err;
        k_m2l<double><<<grid, block, sm, s>>>(e);
    }
    return cudaGetLastError();
}

cudaError_t launch_downward(const EvalBufs& e, bool mixed, int fp64_levels, cudaStream_t s) {
    for (int l = 0; l + 1 < e.n_levels; ++l) {
        cudaError_t err = (!mixed || l < fp64_levels) ? downward_level<double>(e, l, s) : downward_level<float>(e, l, s);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

cudaError_t launch_leaf_eval(const EvalBufs& e, bool mixed, cudaStream_t s) {
    cudaError_t err;
    const int grid = grid_for(e.n_cells, 1, 1 << 20);
    if (mixed) {
        const size_t sm = leaf_smem<float>(e.p, e.nt);
        if ((err = set_smem(k_leaf<float>, sm)) != cudaSuccess) return err;
        k_leaf<float><<<grid, kLeafBlock, sm, s>>>(e);
    } else {
        const size_t sm = leaf_smem<double>(e.p, e.nt);
        if ((err = set_smem(k_leaf<double>, sm)) != cudaSuccess) return err;
        k_leaf<double><<<grid, kLeafBlock, sm, s>>>(e);
    }
    return cudaGetLastError();
}

cudaError_t launch_group(const unsigned long long* list, long long count, int n_cells, int* cnt, int* off, int* cursor,
                         int* src, int* tile_sums, cudaStream_t s) {
    cudaError_t err;
    if ((err = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n_cells, s)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(cursor, 0, sizeof(int) * (size_t)n_cells, s)) != cudaSuccess) return err;
    if (count > 0) k_group_count<<<grid_for(count, 256, 4096), 256, 0, s>>>(list, count, cnt);
    if ((err = scan::exclusive(cnt, off, nullptr, n_cells, tile_sums, off + n_cells, s)) != cudaSuccess) return err;
    if (count > 0) k_group_fill<<<grid_for(count, 256, 4096), 256, 0, s>>>(list, count, off, cursor, src);
    return cudaGetLastError();
}

}  // namespace fmm
}  // namespace gtap
