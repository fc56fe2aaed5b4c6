// Allocation-free block-mode mergesort: gtap_mergesort_noalloc.
//
// Some callers cannot call cudaMalloc: a plugin or library loaded into a host
// application that owns every byte of device memory and hands the plugin only
// a stream and the buffers to work on, a real-time path whose memory budget is
// fixed before it starts, or code running under an allocator that must not be
// re-entered.  For them this entry point keeps every byte of working memory
// the sort needs -- the ping-pong key buffer, the task-record pool, the deques,
// the pool's chunk queue and the control block -- in one file-scope __device__
// array of fixed size, so the call allocates nothing.  The caller passes only
// the input and output.  The call waits for its own stream before returning
// (it reads the device-side status back).
//
// Limits and sharing: at most kNoallocMaxKeys keys per call.  Every GPU that
// loads the library holds the array until the process exits.  All calls share
// it and it keeps the last call's contents; the reset kernel re-initialises
// every part a run reads before writing it, so nothing depends on what a
// previous call left.  Calls whose GPU work overlaps (two streams, or two host
// threads) race on the array and must not be issued.
#include <cstring>

#include <cuda_runtime.h>

#include "gtap.h"
#include "gtap_internal.h"
#include "launch.h"

namespace gtap {
namespace {

constexpr uint64_t kNoallocMaxKeys = 1ull << 20;       // 4 MiB of keys
constexpr uint64_t kNoallocFrames = 1ull << 16;        // 64-byte records: 4 MiB
constexpr int kNoallocMaxBlocks = 160;                 // persistent grid bound (one block per SM on GB300)
constexpr uint32_t kNoallocRing = 1024;                // deque slots per block
constexpr uint64_t kNoallocChunks = 4096;              // chunk-queue slots (>= frames / 32 + 1, power of two)

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffTmp = 0;
constexpr size_t kOffFrames = align256(kOffTmp + kNoallocMaxKeys * 4);
constexpr size_t kOffRings = align256(kOffFrames + kNoallocFrames * 64);
constexpr size_t kOffQs = align256(kOffRings + (size_t)kNoallocMaxBlocks * kNoallocRing * 4);
constexpr size_t kOffCqSeq = align256(kOffQs + (size_t)kNoallocMaxBlocks * sizeof(QState));
constexpr size_t kOffCqIds = align256(kOffCqSeq + kNoallocChunks * 8);
constexpr size_t kOffCtl = align256(kOffCqIds + kNoallocChunks * kChunk * 4);
constexpr size_t kOffRoots = align256(kOffCtl + sizeof(DevControl));
constexpr size_t kOffDesc = align256(kOffRoots + sizeof(RootEntry));
constexpr size_t kOffStats = align256(kOffDesc + sizeof(RootDesc));
constexpr size_t kNoallocBytes = align256(kOffStats + (size_t)kNoallocMaxBlocks * sizeof(WorkerStats));

}  // namespace

// The whole working set of one call.  In host code this name is a host-side
// stand-in: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {

struct DeviceSetup {
    bool done = false;
    char* base = nullptr;       // device address of g_noalloc_scratch on this device
    int grid = 0;
    size_t smem = 0;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];

// Root record writer: the descriptor travels as a kernel argument, so no host
// staging buffer is needed.
__global__ void noalloc_write_root(RootDesc* dst, RootDesc d) { *dst = d; }

gtap_status setup_device(int dev, DeviceSetup* s) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) { cudaGetLastError(); return GTAP_ERR_CUDA; }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GTAP_ERR_CUDA;
    const int bs = 256;
    const int maxspawn = block_kernel_maxspawn(PS_MSORT, bs);
    const size_t smem = (size_t)block_rt_smem(maxspawn) + block_prog_smem(PS_MSORT, bs);
    int occ = 0;
    if (block_kernel_occupancy(PS_MSORT, bs, smem, &occ) != cudaSuccess || occ < 1) return GTAP_ERR_CUDA;
    s->base = static_cast<char*>(p);
    s->grid = sms < kNoallocMaxBlocks ? sms : kNoallocMaxBlocks;
    s->smem = smem;
    s->done = true;
    return GTAP_OK;
}

}  // namespace
}  // namespace gtap

using namespace gtap;

extern "C" gtap_status gtap_mergesort_noalloc(const uint32_t* src, uint32_t* dst, uint64_t n, void* stream) {
    if (n > kNoallocMaxKeys) return GTAP_ERR_INVALID_ARG;
    if (n > 0 && (!src || !dst)) return GTAP_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GTAP_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return GTAP_ERR_INVALID_ARG;
    DeviceSetup& s = g_setup[dev];
    if (!s.done) {
        gtap_status st = setup_device(dev, &s);
        if (st != GTAP_OK) return st;
    }
    if (n == 0) return GTAP_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* b = s.base;

    gtap_mergesort_args a;
    a.src = src;
    a.dst = dst;
    a.tmp = reinterpret_cast<uint32_t*>(b + kOffTmp);
    a.n = n;
    a.leaf = 4096;
    a.merge_cutoff = 16384;
    RootDesc d;
    std::memset(&d, 0, sizeof(d));
    d.type = T_MSORT;
    d.queue = 0;
    struct { uint32_t root, into_tmp; unsigned long long lo, hi; } payload{0u, 0u, 0ull, n};
    std::memcpy(d.payload, &payload, sizeof(payload));
    std::memcpy(d.env, &a, sizeof(a));

    KParams P{};
    P.frames = b + kOffFrames;
    P.n_frames = kNoallocFrames;
    P.frame_bytes = 64;
    P.n_workers = (uint32_t)s.grid;
    P.n_queues = 1;
    P.ring_mask = kNoallocRing - 1;
    P.rings = reinterpret_cast<uint32_t*>(b + kOffRings);
    P.qs = reinterpret_cast<QState*>(b + kOffQs);
    P.cq_seq = reinterpret_cast<unsigned long long*>(b + kOffCqSeq);
    P.cq_ids = reinterpret_cast<uint32_t*>(b + kOffCqIds);
    P.ncq_mask = kNoallocChunks - 1;
    P.ctl = reinterpret_cast<DevControl*>(b + kOffCtl);
    P.roots = reinterpret_cast<RootEntry*>(b + kOffRoots);
    P.root_desc = reinterpret_cast<const RootDesc*>(b + kOffDesc);
    P.n_roots = 1;
    P.maxspawn = (uint32_t)block_kernel_maxspawn(PS_MSORT, 256);
    P.stats = reinterpret_cast<WorkerStats*>(b + kOffStats);
    P.host_abort = nullptr;
    P.timeout_ns = 20ull * 1000000000ull;
    P.seed = 0x5EEDull;
    P.steal_policy = 0;

    noalloc_write_root<<<1, 1, 0, st>>>(reinterpret_cast<RootDesc*>(b + kOffDesc), d);
    if (cudaGetLastError() != cudaSuccess) return GTAP_ERR_CUDA;
    if (launch_reset(P, 1, st) != cudaSuccess) return GTAP_ERR_CUDA;
    if (launch_block_kernel(PS_MSORT, 256, P, s.grid, s.smem, st) != cudaSuccess) { cudaGetLastError(); return GTAP_ERR_CUDA; }
    int code = 0;
    if (cudaMemcpyAsync(&code, &P.ctl->err.code, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GTAP_ERR_CUDA;
    return (gtap_status)code;
}
