// Atomic-rate microbenchmark: the memory-system operations the fork-join
// runtime is built on, measured on this GPU.  Its rates are the ceilings
// against which the thread-mode scheduler kernels are compared.
#include <cuda_runtime.h>

#include "gtap.h"

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// kind 0: scattered atom.add.acq_rel.gpu (value used) on 4-byte words -- the join decrement
// kind 1: scattered red.add (no return) on 8-byte words -- accumulating joins
// kind 2: CAS on one word per warp (lane 0), value used -- deque count claims
// kind 3: CAS on a single word from every warp (lane 0) -- a contended hot word
// kind 4: scattered ld.global.cg of 4-byte words -- L2 round trips
__global__ void k_bench(int kind, unsigned* words, unsigned long long n_words, int iters, unsigned long long* sink) {
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const unsigned long long wid = tid >> 5;
    unsigned long long acc = 0;
    unsigned long long x = tid * 0x9E3779B97F4A7C15ull + 1;
    for (int i = 0; i < iters; ++i) {
        x = mix64(x + i);
        if (kind == 0) {
            unsigned* p = words + (x % n_words);
            unsigned old;
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(0xFFFFFFFFu) : "memory");
            acc += old;
        } else if (kind == 1) {
            unsigned long long* p = reinterpret_cast<unsigned long long*>(words) + (x % (n_words / 2));
            atomicAdd(p, 1ull);
        } else if (kind == 2) {
            if (lane == 0) {
                unsigned* p = words + ((wid * 32) % n_words);
                const unsigned v = __ldcg(p);
                acc += atomicCAS(p, v, v + 1);
            }
        } else if (kind == 3) {
            if (lane == 0) {
                const unsigned v = __ldcg(words);
                acc += atomicCAS(words, v, v + 1);
            }
        } else {
            acc += __ldcg(words + (x % n_words));
        }
    }
    if (acc == 0x123456789ull) *sink = acc;   // keep the results live
}

}  // namespace

extern "C" gtap_status gtap_microbench(int kind, void* region, uint64_t region_bytes, int blocks, int threads, int iters,
                                       float* ms_out, double* ops_out, void* stream) {
    if (kind < 0 || kind > 4 || !region || region_bytes < 4096 || blocks < 1 || threads < 32 || threads > 1024 ||
        threads % 32 || iters < 1 || !ms_out || !ops_out)
        return GTAP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return GTAP_ERR_CUDA;
    unsigned* words = static_cast<unsigned*>(region);
    const unsigned long long n_words = (region_bytes - 64) / 4;
    unsigned long long* sink = reinterpret_cast<unsigned long long*>(static_cast<char*>(region) + region_bytes - 64);
    k_bench<<<blocks, threads, 0, s>>>(kind, words, n_words, 1, sink);   // warm-up
    cudaEventRecord(a, s);
    k_bench<<<blocks, threads, 0, s>>>(kind, words, n_words, iters, sink);
    cudaEventRecord(b, s);
    gtap_status st = GTAP_OK;
    if (cudaEventSynchronize(b) != cudaSuccess) st = GTAP_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double per_thread = (kind == 2 || kind == 3) ? 1.0 / 32.0 : 1.0;
    *ms_out = ms;
    *ops_out = (double)blocks * threads * per_thread * iters;
    return st;
}
