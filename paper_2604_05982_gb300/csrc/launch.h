// Host-side entry points of the kernel translation units (internal).
#pragma once
#include <cuda_runtime.h>
#include "gtap_internal.h"
#include "gtap.h"

namespace gtap {

// Thread mode: persistent scheduler kernel for a program set.
// sched: GTAP_SCHED_* (the comparison variants exist for fib, N-Queens, the hashed tree and the binary tree).
cudaError_t launch_thread_kernel(unsigned pset, int sched, const KParams& P, int grid, int block, size_t smem,
                                 cudaStream_t s);
cudaError_t thread_kernel_occupancy(unsigned pset, int sched, int block, size_t smem, int* blocks_per_sm);
unsigned thread_kernel_pset(unsigned registered);   // instantiation that covers the registered programs
int thread_kernel_maxspawn(unsigned pset);
size_t thread_prog_smem(unsigned pset);             // per-warp shared bytes the programs of the set use
uint32_t thread_record_bytes(unsigned pset);

// Block mode (block size 128 or 256).
cudaError_t launch_block_kernel(unsigned pset, int bs, const KParams& P, int grid, size_t smem, cudaStream_t s);
cudaError_t block_kernel_occupancy(unsigned pset, int bs, size_t smem, int* blocks_per_sm);
unsigned block_kernel_pset(unsigned registered);
int block_kernel_maxspawn(unsigned pset, int bs);
size_t block_prog_smem(unsigned pset, int bs);
uint32_t block_record_bytes(unsigned pset, int bs);

// Re-zero deques, pool, control words; write root records and push them.
cudaError_t launch_reset(const KParams& P, int init_chunk_queue, cudaStream_t s);

}  // namespace gtap

extern "C" gtap_status gtap_debug_record_log(gtap_ctx* c, uint32_t id, uint64_t* out);
