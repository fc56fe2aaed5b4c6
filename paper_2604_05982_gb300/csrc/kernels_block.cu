// Block-mode persistent kernels, one instantiation per program set and block size.
#include "launch.h"
#include "gtap_device.cuh"
#include "programs_block.cuh"
#include "programs_dtt.cuh"
#include "programs_micro.cuh"

namespace gtap {

template <unsigned PSET, int BS>
struct BlockDispatch {
    __device__ static void run(BTaskCtx& c) {
        switch (c.type()) {
        case T_MSORT:
            if constexpr ((PSET & PS_MSORT) != 0) { msort_step<BS>(c); return; }
            break;
        case T_MMERGE:
            if constexpr ((PSET & PS_MSORT) != 0) { mmerge_step<BS>(c); return; }
            break;
        case T_INTEGRATE_BLK:
            if constexpr ((PSET & PS_INTEGRATE_BLK) != 0) { integrate_blk_step<BS>(c); return; }
            break;
        case T_DTT:
            if constexpr ((PSET & PS_DTT) != 0) { dtt_step<BS>(c); return; }
            break;
        case T_BINTREE_BLK:
            if constexpr ((PSET & PS_BINTREE_BLK) != 0) { bintree_blk_step<BS>(c); return; }
            break;
        default:
            break;
        }
        if (threadIdx.x == 0) c.fail(GTAP_ERR_UNKNOWN_TASK, (unsigned long long)c.type());
    }
};

template <unsigned PSET, int BS>
__global__ void __launch_bounds__(BS, 768 / BS) block_kernel(KParams P) {
    extern __shared__ __align__(16) char smem[];
    block_mode_loop<BlockDispatch<PSET, BS>>(P, smem, BS);
}

constexpr unsigned PS_BLOCK_ALL = PS_MSORT | PS_INTEGRATE_BLK | PS_DTT | PS_BINTREE_BLK;
// The binary-tree microbenchmark also runs with one-warp blocks (Sec. 6.1 uses block size 32 in both modes).
#define GTAP_BLOCK_SETS(X) X(PS_MSORT, 256) X(PS_INTEGRATE_BLK, 256) X(PS_DTT, 256) X(PS_BLOCK_ALL, 256) \
                           X(PS_MSORT, 128) X(PS_INTEGRATE_BLK, 128) X(PS_DTT, 128) X(PS_BLOCK_ALL, 128) \
                           X(PS_BINTREE_BLK, 256) X(PS_BINTREE_BLK, 128) X(PS_BINTREE_BLK, 32)

static const void* block_kernel_fn(unsigned pset, int bs) {
#define X(S, B) if (pset == (S) && bs == (B)) return reinterpret_cast<const void*>(&block_kernel<(S), (B)>);
    GTAP_BLOCK_SETS(X)
#undef X
    return nullptr;
}

unsigned block_kernel_pset(unsigned registered) {
    const unsigned singles[] = {PS_MSORT, PS_INTEGRATE_BLK, PS_DTT, PS_BINTREE_BLK};
    for (unsigned s : singles)
        if (registered != 0 && (registered & ~s) == 0) return s;
    return PS_BLOCK_ALL;
}

// Most children one block step can spawn: a forked merge spawns one piece per
// thread, a traversal task one child per kDttGroup frontier pairs.
int block_kernel_maxspawn(unsigned pset, int bs) {
    int m = 2;
    if (pset & PS_MSORT) m = std::max(m, bs);
    if (pset & PS_DTT) m = std::max(m, kDttMaxSpawn + 1);
    return m;
}

size_t block_prog_smem(unsigned pset, int bs) {
    size_t b = 0;
    if (pset & PS_MSORT) b = std::max(b, (size_t)(kMsStages * kMsStride * 4 + 8 * 260));
    if (pset & PS_INTEGRATE_BLK) b = std::max(b, (size_t)(8 * bs));
    if (pset & PS_DTT) b = std::max(b, sizeof(DttShared) + 16);
    if (pset & PS_BINTREE_BLK) b = std::max(b, (size_t)(8 * 32));
    return b;
}

uint32_t block_record_bytes(unsigned pset, int bs) {
    uint32_t r = 64;
    if (pset & PS_INTEGRATE_BLK) r = std::max<uint32_t>(r, bs == 128 ? integ_blk_record<128>() : integ_blk_record<256>());
    if (pset & PS_DTT) r = std::max<uint32_t>(r, (uint32_t)(kHdrBytes + sizeof(fmm::DttSpawn)));
    return (r + 63u) & ~63u;
}

cudaError_t launch_block_kernel(unsigned pset, int bs, const KParams& P, int grid, size_t smem, cudaStream_t s) {
    const void* fn = block_kernel_fn(pset, bs);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<KParams*>(&P)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(bs), args, smem, s);
}

cudaError_t block_kernel_occupancy(unsigned pset, int bs, size_t smem, int* blocks_per_sm) {
    const void* fn = block_kernel_fn(pset, bs);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, bs, smem);
}

}  // namespace gtap
