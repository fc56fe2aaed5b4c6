// Thread-mode persistent kernels, one instantiation per program set.
#include "launch.h"
#include "gtap_device.cuh"
#include "programs_thread.cuh"
#include "programs_micro.cuh"

namespace gtap {

template <unsigned PSET>
struct ThreadDispatch {
    __device__ static void run(TaskCtx& c) {
        switch (c.type()) {
        case T_FIB:
            if constexpr ((PSET & PS_FIB) != 0) { fib_step(c); return; }
            break;
        case T_NQUEENS:
            if constexpr ((PSET & PS_NQUEENS) != 0) { nqueens_step(c); return; }
            break;
        case T_UTS:
            if constexpr ((PSET & PS_UTS) != 0) { uts_step(c); return; }
            break;
        case T_UTS_RANGE:
            if constexpr ((PSET & PS_UTS) != 0) { uts_range_step(c); return; }
            break;
        case T_INTEGRATE:
            if constexpr ((PSET & PS_INTEGRATE) != 0) { integrate_step(c); return; }
            break;
        case T_KCLIQUE_ROOT:
            if constexpr ((PSET & PS_KCLIQUE) != 0) { kclique_range_step(c); return; }
            break;
        case T_KCLIQUE_SET:
            if constexpr ((PSET & PS_KCLIQUE) != 0) { kclique_set_dispatch(c); return; }
            break;
        case T_KCLIQUE_PIV:
            if constexpr ((PSET & PS_KCLIQUE) != 0) { kclique_piv_step(c); return; }
            break;
        case T_KCLIQUE_PIVB:
            if constexpr ((PSET & PS_KCLIQUE) != 0) { kclique_pivb_step(c); return; }
            break;
        case T_BINTREE:
            if constexpr ((PSET & PS_BINTREE) != 0) { bintree_step(c); return; }
            break;
        case T_TSORT:
            if constexpr ((PSET & PS_CILKSORT) != 0) { cilksort_sort_step(c); return; }
            break;
        case T_TMERGE:
            if constexpr ((PSET & PS_CILKSORT) != 0) { cilksort_merge_step(c); return; }
            break;
        default:
            break;
        }
        c.fail(GTAP_ERR_UNKNOWN_TASK, (unsigned long long)c.type());
        // drop the task: completing it would touch a record of unknown layout
    }
};

// Resident 256-thread blocks per SM each program set is compiled for (the
// register budget follows): k-clique tasks wait on L2 round trips, so it keeps
// 4 blocks (64 registers); N-Queens and the full set measured faster with 80
// registers at 3 blocks than capped at 64.
template <unsigned PSET>
constexpr int thread_min_blocks() {
    return (PSET == PS_NQUEENS || PSET == PS_THREAD_ALL) ? 3 : 4;
}

template <unsigned PSET, int SCHED>
__global__ void __launch_bounds__(256, thread_min_blocks<PSET>()) thread_kernel(KParams P) {
    extern __shared__ __align__(16) char smem[];
    const int wib = threadIdx.x >> 5;
    thread_mode_loop<ThreadDispatch<PSET>, SCHED>(P, smem + (size_t)wib * P.warp_smem);
}

// Default scheduler for every program set; the Sec. 6.5 comparison variants for
// the scheduler-bound microbenchmark programs.
#define GTAP_THREAD_SETS(X)                                                                                       \
    X(PS_FIB, SCHED_BATCHED) X(PS_NQUEENS, SCHED_BATCHED) X(PS_UTS, SCHED_BATCHED) X(PS_INTEGRATE, SCHED_BATCHED) \
    X(PS_KCLIQUE, SCHED_BATCHED) X(PS_BINTREE, SCHED_BATCHED) X(PS_CILKSORT, SCHED_BATCHED)                       \
    X(PS_THREAD_ALL, SCHED_BATCHED)                                                                               \
    X(PS_FIB, SCHED_GLOBAL) X(PS_FIB, SCHED_SINGLE) X(PS_UTS, SCHED_GLOBAL) X(PS_UTS, SCHED_SINGLE)               \
    X(PS_BINTREE, SCHED_GLOBAL) X(PS_BINTREE, SCHED_SINGLE)

static const void* thread_kernel_fn(unsigned pset, int sched) {
#define X(S, Q) if (pset == (S) && sched == (Q)) return reinterpret_cast<const void*>(&thread_kernel<(S), (Q)>);
    GTAP_THREAD_SETS(X)
#undef X
    return nullptr;
}

unsigned thread_kernel_pset(unsigned registered) {
    const unsigned singles[] = {PS_FIB, PS_NQUEENS, PS_UTS, PS_INTEGRATE, PS_KCLIQUE, PS_BINTREE, PS_CILKSORT};
    for (unsigned s : singles)
        if (registered != 0 && (registered & ~s) == 0) return s;
    return PS_THREAD_ALL;
}

int thread_kernel_maxspawn(unsigned pset) {
    int m = 1;
    if (pset & PS_FIB) m = max(m, 2);
    if (pset & PS_NQUEENS) m = max(m, 16);
    if (pset & PS_UTS) m = max(m, 8);
    if (pset & PS_INTEGRATE) m = max(m, 2);
    if (pset & PS_KCLIQUE) m = max(m, kKcFan);
    if (pset & PS_BINTREE) m = max(m, 2);
    if (pset & PS_CILKSORT) m = max(m, 2);
    return m;
}

size_t thread_prog_smem(unsigned pset) { return (pset & PS_KCLIQUE) ? (size_t)kKcCoopSmem : 0; }

uint32_t thread_record_bytes(unsigned) { return 64; }

cudaError_t launch_thread_kernel(unsigned pset, int sched, const KParams& P, int grid, int block, size_t smem,
                                 cudaStream_t s) {
    const void* fn = thread_kernel_fn(pset, sched);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<KParams*>(&P)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, s);
}

cudaError_t thread_kernel_occupancy(unsigned pset, int sched, int block, size_t smem, int* blocks_per_sm) {
    const void* fn = thread_kernel_fn(pset, sched);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

}  // namespace gtap
