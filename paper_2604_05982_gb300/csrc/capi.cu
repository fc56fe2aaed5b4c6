// Host runtime behind the C ABI (include/gtap.h): context, storage, root
// queueing, launch, bounded wait, result and statistics readback.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "gtap.h"
#include "gtap_internal.h"
#include "launch.h"
#include "fmm_internal.h"

using namespace gtap;

namespace {

struct ProgInfo {
    const char* name;
    gtap_mode mode;
    int type;
    unsigned pset;
};
const ProgInfo kPrograms[] = {
    {"fib", GTAP_MODE_THREAD, T_FIB, PS_FIB},
    {"nqueens", GTAP_MODE_THREAD, T_NQUEENS, PS_NQUEENS},
    {"uts", GTAP_MODE_THREAD, T_UTS, PS_UTS},
    {"integrate", GTAP_MODE_THREAD, T_INTEGRATE, PS_INTEGRATE},
    {"kclique", GTAP_MODE_THREAD, T_KCLIQUE_ROOT, PS_KCLIQUE},
    {"mergesort", GTAP_MODE_BLOCK, T_MSORT, PS_MSORT},
    {"integrate_block", GTAP_MODE_BLOCK, T_INTEGRATE_BLK, PS_INTEGRATE_BLK},
    {"fmm_dtt", GTAP_MODE_BLOCK, T_DTT, PS_DTT},
    {"bintree", GTAP_MODE_THREAD, T_BINTREE, PS_BINTREE},
    {"cilksort", GTAP_MODE_THREAD, T_TSORT, PS_CILKSORT},
    {"bintree_block", GTAP_MODE_BLOCK, T_BINTREE_BLK, PS_BINTREE_BLK},
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
uint32_t next_pow2(uint32_t v) {
    uint32_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

struct gtap_ctx {
    gtap_mode mode = GTAP_MODE_THREAD;
    int n_queues = 1;
    size_t pool_bytes = 0;
    gtap_config cfg{};
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr;
    int threads_per_block = 256, blocks_per_sm = 4, grid = 0;
    uint32_t n_workers_max = 0, ring_cap = 0;
    uint64_t ncq = 0;

    bool own_arena = false;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    char* frames = nullptr;
    uint32_t* rings = nullptr;
    QState* qs = nullptr;
    unsigned long long* cq_seq = nullptr;
    uint32_t* cq_ids = nullptr;
    DevControl* ctl = nullptr;
    RootEntry* roots = nullptr;
    RootDesc* root_desc = nullptr;
    WorkerStats* stats = nullptr;
    char* scratch = nullptr;
    unsigned long long* sq_seq = nullptr;
    uint32_t* sq_ids = nullptr;
    uint64_t sq_mask = 0;
    unsigned long long* lq_seq = nullptr;
    uint32_t* lq_ids = nullptr;
    uint64_t lq_mask = 0;
    char* blocks = nullptr;
    uint64_t blocks_bytes = 0;
    unsigned* fstate = nullptr;
    unsigned long long* flog = nullptr;
    unsigned* flogn = nullptr;
    uint64_t max_frames = 0;
    unsigned long long* gq = nullptr;   // central-queue scheduler slots
    uint64_t gq_cap = 0;

    RootDesc* root_desc_pinned = nullptr;
    int* host_abort = nullptr;       // pinned, mapped
    int* host_abort_dev = nullptr;
    DevControl* ctl_pinned = nullptr;
    RootEntry* roots_pinned = nullptr;
    WorkerStats* stats_pinned = nullptr;

    std::vector<RootDesc> pending_roots;
    unsigned registered = 0;
    bool registered_type[T_MAX] = {};

    // last launch
    bool running = false;
    bool have_results = false;
    uint32_t launched_roots = 0;
    uint32_t launched_workers = 0;
    int launched_grid = 0;
    uint64_t launched_frames = 0;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;   // whole run (root upload, reset, kernel)
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;         // the persistent kernel alone
    gtap_stats last_stats{};
    gtap_error_info last_err{};
    bool cq_initialised = false;
    // CUDA-graph replay of a captured run
    cudaStream_t own_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool graph_valid = false;
    uint32_t graph_roots = 0, graph_workers = 0;
    int graph_grid = 0;
    uint64_t graph_frames = 0;
    cudaStream_t run_stream = nullptr;   // stream of the launch in flight
    // serving
    bool serving = false;
    InboxSlot* inbox = nullptr;          // mapped pinned
    OutboxEntry* outbox = nullptr;
    HostFlags* hflags = nullptr;
    InboxSlot* inbox_dev = nullptr;
    OutboxEntry* outbox_dev = nullptr;
    HostFlags* hflags_dev = nullptr;
    uint64_t submitted = 0;
};

extern "C" {

const char* gtap_status_string(gtap_status s) {
    switch (s) {
    case GTAP_OK: return "ok";
    case GTAP_ERR_INVALID_ARG: return "invalid argument";
    case GTAP_ERR_NO_MEMORY: return "out of memory";
    case GTAP_ERR_POOL_EXHAUSTED: return "task-record pool exhausted";
    case GTAP_ERR_DEQUE_OVERFLOW: return "deque overflow";
    case GTAP_ERR_LIST_OVERFLOW: return "interaction list overflow";
    case GTAP_ERR_TIMEOUT: return "timeout";
    case GTAP_ERR_CUDA: return "CUDA error";
    case GTAP_ERR_BUSY: return "run in flight";
    case GTAP_ERR_UNKNOWN_TASK: return "unknown task type";
    case GTAP_ERR_TASK_FAILED: return "task failed";
    case GTAP_ERR_NOT_READY: return "result not ready";
    }
    return "unknown status";
}

static void drop_graph(gtap_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_valid = false;
}

static gtap_status free_all(gtap_ctx* c) {
    drop_graph(c);
    if (c->inbox) cudaFreeHost(c->inbox);
    if (c->outbox) cudaFreeHost(c->outbox);
    if (c->hflags) cudaFreeHost(c->hflags);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    if (c->own_arena && c->arena) cudaFree(c->arena);
    if (c->root_desc_pinned) cudaFreeHost(c->root_desc_pinned);
    if (c->host_abort) cudaFreeHost(c->host_abort);
    if (c->ctl_pinned) cudaFreeHost(c->ctl_pinned);
    if (c->roots_pinned) cudaFreeHost(c->roots_pinned);
    if (c->stats_pinned) cudaFreeHost(c->stats_pinned);
    if (c->ev_start) cudaEventDestroy(c->ev_start);
    if (c->ev_stop) cudaEventDestroy(c->ev_stop);
    if (c->ev_k0) cudaEventDestroy(c->ev_k0);
    if (c->ev_k1) cudaEventDestroy(c->ev_k1);
    delete c;
    return GTAP_OK;
}

// Launch geometry and arena layout of a context (shared by gtap_init and gtap_arena_bytes).
struct ArenaLayout {
    int threads_per_block = 256, blocks_per_sm = 4, grid = 0;
    uint32_t ring_cap = 0, n_workers_max = 0;
    uint64_t ncq = 0, max_frames = 0;
    size_t o_frames = 0, o_rings = 0, o_qs = 0, o_cqs = 0, o_cqi = 0, o_ctl = 0, o_roots = 0, o_desc = 0,
           o_stats = 0, o_scratch = 0, o_fstate = 0, o_flog = 0, o_flogn = 0, o_gq = 0, total = 0;
    uint64_t gq_cap = 0;
};

// Validates the arguments, fills the defaults of cfg in place and computes the layout.
static gtap_status plan_arena(gtap_mode mode, int n_queues, size_t frame_pool_bytes, gtap_config& cfg, int sm_count,
                              ArenaLayout* L) {
    if (mode != GTAP_MODE_THREAD && mode != GTAP_MODE_BLOCK) return GTAP_ERR_INVALID_ARG;
    if (n_queues < 1 || n_queues > kMaxQueues) return GTAP_ERR_INVALID_ARG;
    if (mode == GTAP_MODE_BLOCK && n_queues != 1) return GTAP_ERR_INVALID_ARG;
    if (frame_pool_bytes < 64 * 1024) return GTAP_ERR_INVALID_ARG;
    if (mode == GTAP_MODE_THREAD) {
        L->threads_per_block = cfg.threads_per_block ? cfg.threads_per_block : 256;
        if (L->threads_per_block < 32 || L->threads_per_block > 256 || L->threads_per_block % 32) return GTAP_ERR_INVALID_ARG;
        L->blocks_per_sm = cfg.blocks_per_sm ? cfg.blocks_per_sm : 4;
        L->ring_cap = cfg.deque_capacity ? (uint32_t)cfg.deque_capacity : 4096u;
    } else {
        L->threads_per_block = cfg.threads_per_block ? cfg.threads_per_block : 256;
        // 32 (one warp per block) is instantiated for the binary-tree microbenchmark only
        if (L->threads_per_block != 32 && L->threads_per_block != 128 && L->threads_per_block != 256)
            return GTAP_ERR_INVALID_ARG;
        L->blocks_per_sm = cfg.blocks_per_sm ? cfg.blocks_per_sm : 4;
        L->ring_cap = cfg.deque_capacity ? (uint32_t)cfg.deque_capacity : 1024u;
    }
    if (L->blocks_per_sm < 1 || L->blocks_per_sm > 32) return GTAP_ERR_INVALID_ARG;
    if (L->ring_cap < 32 || next_pow2(L->ring_cap) != L->ring_cap || L->ring_cap > (1u << 24)) return GTAP_ERR_INVALID_ARG;
    if (cfg.frame_bytes != 0 && cfg.frame_bytes != 64 && cfg.frame_bytes != 128) return GTAP_ERR_INVALID_ARG;
    if (!cfg.max_roots) cfg.max_roots = 4096;
    if (cfg.max_roots < 1 || cfg.max_roots > (1 << 24)) return GTAP_ERR_INVALID_ARG;
    if (!cfg.timeout_ns) cfg.timeout_ns = 60ull * 1000000000ull;
    if (!cfg.seed) cfg.seed = 0x5EEDull;
    if (!cfg.idle_backoff_ns) cfg.idle_backoff_ns = 512;
    if (cfg.idle_backoff_ns < 32 || cfg.idle_backoff_ns > 65536) return GTAP_ERR_INVALID_ARG;
    if (cfg.grid_blocks < 0) return GTAP_ERR_INVALID_ARG;
    if (cfg.scheduler < 0 || cfg.scheduler > 2) return GTAP_ERR_INVALID_ARG;
    // the scheduler comparison variants are thread-mode designs with one queue per warp
    if (cfg.scheduler != 0 && (mode != GTAP_MODE_THREAD || n_queues != 1)) return GTAP_ERR_INVALID_ARG;
    L->grid = L->blocks_per_sm * sm_count;
    if (cfg.grid_blocks > 0) L->grid = std::min(cfg.grid_blocks, L->grid);
    L->n_workers_max = (mode == GTAP_MODE_THREAD) ? (uint32_t)(L->grid * (L->threads_per_block / 32)) : (uint32_t)L->grid;

    // storage layout (256-byte aligned pieces of one arena)
    const uint64_t max_frames = frame_pool_bytes / 64;
    L->max_frames = max_frames;
    L->ncq = next_pow2((uint32_t)std::min<uint64_t>((max_frames + kChunk - 1) / kChunk + 1, 1ull << 31));
    const size_t qn = (size_t)L->n_workers_max * n_queues;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L->o_frames = take(frame_pool_bytes);
    L->o_rings = take(qn * L->ring_cap * sizeof(uint32_t));
    L->o_qs = take(qn * sizeof(QState));
    L->o_cqs = take(L->ncq * sizeof(unsigned long long));
    L->o_cqi = take(L->ncq * kChunk * sizeof(uint32_t));
    L->o_ctl = take(sizeof(DevControl));
    L->o_roots = take((size_t)cfg.max_roots * sizeof(RootEntry));
    L->o_desc = take((size_t)cfg.max_roots * sizeof(RootDesc));
    L->o_stats = take((size_t)L->n_workers_max * sizeof(WorkerStats));
    L->o_scratch = take(cfg.scratch_bytes);
    L->o_fstate = take(cfg.debug_checks ? (size_t)max_frames * sizeof(unsigned) : 0);
    L->o_flog = take(cfg.debug_checks > 1 ? (size_t)max_frames * 8 * sizeof(unsigned long long) : 0);
    L->o_flogn = take(cfg.debug_checks > 1 ? (size_t)max_frames * sizeof(unsigned) : 0);
    // central queue: one slot per record, so it never fills
    L->gq_cap = cfg.scheduler == GTAP_SCHED_GLOBAL ? next_pow2((uint32_t)std::min<uint64_t>(max_frames, 1ull << 31)) : 0;
    L->o_gq = take(L->gq_cap * sizeof(unsigned long long));
    L->total = off;
    return GTAP_OK;
}

gtap_status gtap_arena_bytes(gtap_mode mode, int n_queues, size_t frame_pool_bytes, const gtap_config* cfg_in,
                             size_t* out) {
    if (!out) return GTAP_ERR_INVALID_ARG;
    *out = 0;
    gtap_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return GTAP_ERR_CUDA;
    }
    ArenaLayout L;
    gtap_status st = plan_arena(mode, n_queues, frame_pool_bytes, cfg, sms, &L);
    if (st != GTAP_OK) return st;
    *out = L.total;
    return GTAP_OK;
}

gtap_status gtap_init(gtap_mode mode, int n_queues, size_t frame_pool_bytes, const gtap_config* cfg_in, gtap_ctx** out) {
    if (!out) return GTAP_ERR_INVALID_ARG;
    *out = nullptr;
    gtap_ctx* c = new gtap_ctx();
    c->mode = mode;
    c->n_queues = n_queues;
    c->pool_bytes = frame_pool_bytes;
    if (cfg_in) c->cfg = *cfg_in;
    gtap_config& cfg = c->cfg;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return GTAP_ERR_CUDA;
    }
    ArenaLayout L;
    {
        gtap_status st = plan_arena(mode, n_queues, frame_pool_bytes, cfg, c->sm_count, &L);
        if (st != GTAP_OK) { delete c; return st; }
    }
    c->threads_per_block = L.threads_per_block;
    c->blocks_per_sm = L.blocks_per_sm;
    c->ring_cap = L.ring_cap;
    c->stream = reinterpret_cast<cudaStream_t>(cfg.stream);
    c->grid = L.grid;
    c->n_workers_max = L.n_workers_max;
    c->ncq = L.ncq;
    const uint64_t max_frames = L.max_frames;
    const size_t o_frames = L.o_frames, o_rings = L.o_rings, o_qs = L.o_qs, o_cqs = L.o_cqs, o_cqi = L.o_cqi,
                 o_ctl = L.o_ctl, o_roots = L.o_roots, o_desc = L.o_desc, o_stats = L.o_stats,
                 o_scratch = L.o_scratch, o_fstate = L.o_fstate, o_flog = L.o_flog, o_flogn = L.o_flogn;
    const size_t total = L.total;

    if (cfg.device_arena) {
        if (cfg.arena_bytes < total || (reinterpret_cast<uintptr_t>(cfg.device_arena) & 255u)) { delete c; return GTAP_ERR_NO_MEMORY; }
        c->arena = static_cast<char*>(cfg.device_arena);
        c->own_arena = false;
    } else {
        if (cudaMalloc(&c->arena, total) != cudaSuccess) { cudaGetLastError(); delete c; return GTAP_ERR_NO_MEMORY; }
        c->own_arena = true;
    }
    c->arena_bytes = total;
    c->frames = c->arena + o_frames;
    c->rings = reinterpret_cast<uint32_t*>(c->arena + o_rings);
    c->qs = reinterpret_cast<QState*>(c->arena + o_qs);
    c->cq_seq = reinterpret_cast<unsigned long long*>(c->arena + o_cqs);
    c->cq_ids = reinterpret_cast<uint32_t*>(c->arena + o_cqi);
    c->ctl = reinterpret_cast<DevControl*>(c->arena + o_ctl);
    c->roots = reinterpret_cast<RootEntry*>(c->arena + o_roots);
    c->root_desc = reinterpret_cast<RootDesc*>(c->arena + o_desc);
    c->stats = reinterpret_cast<WorkerStats*>(c->arena + o_stats);
    c->scratch = cfg.scratch_bytes ? c->arena + o_scratch : nullptr;
    if (c->scratch) {
        // the free-block queue sits at the front of the scratch arena, the blocks after it
        const uint64_t nb0 = cfg.scratch_bytes / kScratchBlock;
        if (nb0 < 2) { free_all(c); return GTAP_ERR_INVALID_ARG; }
        const uint64_t nq = next_pow2((uint32_t)std::min<uint64_t>(nb0 + 1, 1ull << 31));
        // the large-chunk queue after it: one slot per chunk the arena can hold
        const uint64_t nlq = next_pow2((uint32_t)std::min<uint64_t>(nb0 / kScratchLargeBlocks + 1, 1ull << 31));
        const size_t slot = sizeof(unsigned long long) + sizeof(uint32_t);
        const uint64_t qbytes = align_up((nq + nlq) * slot, kScratchBlock);
        if (qbytes + kScratchBlock > cfg.scratch_bytes) { free_all(c); return GTAP_ERR_INVALID_ARG; }
        c->sq_seq = reinterpret_cast<unsigned long long*>(c->scratch);
        c->sq_ids = reinterpret_cast<uint32_t*>(c->scratch + nq * sizeof(unsigned long long));
        c->sq_mask = nq - 1;
        c->lq_seq = reinterpret_cast<unsigned long long*>(c->scratch + nq * slot);
        c->lq_ids = reinterpret_cast<uint32_t*>(c->scratch + nq * slot + nlq * sizeof(unsigned long long));
        c->lq_mask = nlq - 1;
        c->blocks = c->scratch + qbytes;
        c->blocks_bytes = (cfg.scratch_bytes - qbytes) / kScratchBlock * kScratchBlock;
    }
    c->fstate = cfg.debug_checks ? reinterpret_cast<unsigned*>(c->arena + o_fstate) : nullptr;
    c->flog = cfg.debug_checks > 1 ? reinterpret_cast<unsigned long long*>(c->arena + o_flog) : nullptr;
    c->flogn = cfg.debug_checks > 1 ? reinterpret_cast<unsigned*>(c->arena + o_flogn) : nullptr;
    c->max_frames = max_frames;
    c->gq_cap = L.gq_cap;
    c->gq = L.gq_cap ? reinterpret_cast<unsigned long long*>(c->arena + L.o_gq) : nullptr;

    bool ok = cudaHostAlloc(reinterpret_cast<void**>(&c->root_desc_pinned), (size_t)cfg.max_roots * sizeof(RootDesc), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(reinterpret_cast<void**>(&c->host_abort), 128, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->host_abort_dev), c->host_abort, 0) == cudaSuccess &&
              cudaHostAlloc(reinterpret_cast<void**>(&c->ctl_pinned), sizeof(DevControl), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(reinterpret_cast<void**>(&c->roots_pinned), (size_t)cfg.max_roots * sizeof(RootEntry), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(reinterpret_cast<void**>(&c->stats_pinned), (size_t)c->n_workers_max * sizeof(WorkerStats), cudaHostAllocDefault) == cudaSuccess &&
              cudaEventCreate(&c->ev_start) == cudaSuccess && cudaEventCreate(&c->ev_stop) == cudaSuccess &&
              cudaEventCreate(&c->ev_k0) == cudaSuccess && cudaEventCreate(&c->ev_k1) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        return GTAP_ERR_NO_MEMORY;
    }
    *c->host_abort = 0;
    if (cudaMemset(c->ctl, 0, sizeof(DevControl)) != cudaSuccess) { free_all(c); return GTAP_ERR_CUDA; }
    *out = c;
    return GTAP_OK;
}

gtap_status gtap_register_task(gtap_ctx* c, const char* program, int* out_type) {
    if (!c || !program || !out_type) return GTAP_ERR_INVALID_ARG;
    for (const ProgInfo& p : kPrograms) {
        if (std::strcmp(p.name, program) == 0) {
            if (p.mode != c->mode) return GTAP_ERR_INVALID_ARG;
            c->registered |= p.pset;
            c->registered_type[p.type] = true;
            *out_type = p.type;
            return GTAP_OK;
        }
    }
    return GTAP_ERR_INVALID_ARG;
}

// Translate a program's public argument struct into the root record payload
// and the read-only per-root environment.
static gtap_status make_root(gtap_ctx* c, int type, const void* args, size_t nbytes, int queue, uint32_t root_index,
                             RootDesc* d) {
    std::memset(d, 0, sizeof(*d));
    d->type = (uint32_t)type;
    d->queue = (uint32_t)queue;
    auto put = [&](const void* src, size_t n) { std::memcpy(d->payload, src, n); };
    switch (type) {
    case T_FIB: {
        if (nbytes != sizeof(gtap_fib_args)) return GTAP_ERR_INVALID_ARG;
        gtap_fib_args a;
        std::memcpy(&a, args, sizeof(a));
        if (a.n < 0 || a.n > 92 || a.cutoff < 0 || a.cutoff > 63) return GTAP_ERR_INVALID_ARG;
        int32_t p[2] = {a.n, (a.route ? 1 : 0) | (a.cutoff << 8)};
        put(p, sizeof(p));
        return GTAP_OK;
    }
    case T_NQUEENS: {
        if (nbytes != sizeof(gtap_nqueens_args)) return GTAP_ERR_INVALID_ARG;
        gtap_nqueens_args a;
        std::memcpy(&a, args, sizeof(a));
        if (a.n < 1 || a.n > 16 || a.route < 0 || a.route > 2 || a.cutoff < 0 || a.cutoff > 16)
            return GTAP_ERR_INVALID_ARG;
        uint32_t p[8] = {0, 0, 0, (uint32_t)(0 | (a.n << 8) | ((uint32_t)a.route << 16) | ((uint32_t)a.cutoff << 24)),
                         0, 0, 0, 0};
        put(p, sizeof(p));
        return GTAP_OK;
    }
    case T_UTS: {
        if (nbytes != sizeof(gtap_uts_args)) return GTAP_ERR_INVALID_ARG;
        gtap_uts_args a;
        std::memcpy(&a, args, sizeof(a));
        if (a.m > 8 || a.root_children == 0xFFFFFFFFu) return GTAP_ERR_INVALID_ARG;
        // payload: id = seed (hashed on the device: kUtsHashRoot), threshold, m | route << 8 | flag, arity, acc
        struct { unsigned long long id, thr; uint32_t m_route, arity; unsigned long long acc; } p;
        p.id = a.seed;
        p.thr = a.threshold;
        p.m_route = a.m | ((a.route ? 1u : 0u) << 8) | (1u << 16);
        p.arity = a.root_children;
        p.acc = 0;
        put(&p, sizeof(p));
        return GTAP_OK;
    }
    case T_INTEGRATE: {
        if (nbytes != sizeof(gtap_integrate_args)) return GTAP_ERR_INVALID_ARG;
        gtap_integrate_args a;
        std::memcpy(&a, args, sizeof(a));
        if (!(a.eps > 0.0)) return GTAP_ERR_INVALID_ARG;
        double p[4] = {a.a, a.b, a.eps, 0.0};
        put(p, sizeof(p));
        return GTAP_OK;
    }
    case T_KCLIQUE_ROOT: {
        if (nbytes != sizeof(gtap_kclique_args)) return GTAP_ERR_INVALID_ARG;
        gtap_kclique_args a;
        std::memcpy(&a, args, sizeof(a));
        if (a.split_threshold == 0) a.split_threshold = 64;
        if (a.k < 3 || a.k > 16 || a.split_threshold < 2 || a.split_threshold > 64 || a.edge_begin < 0 ||
            a.algorithm < 0 || a.algorithm > 1 ||
            a.edge_end < a.edge_begin || a.edge_end >= (1ll << 32) ||
            (a.edge_end > a.edge_begin && (!a.off || !a.adj || !a.src)))
            return GTAP_ERR_INVALID_ARG;
        struct { uint32_t root, lo, hi, pad; unsigned long long acc, local; } p{
            root_index, (uint32_t)a.edge_begin, (uint32_t)a.edge_end, 0u, 0ull, 0ull};
        put(&p, sizeof(p));
        std::memcpy(d->env, &a, sizeof(a));
        return GTAP_OK;
    }
    case T_BINTREE:
    case T_BINTREE_BLK: {
        if (nbytes != sizeof(gtap_bintree_args)) return GTAP_ERR_INVALID_ARG;
        gtap_bintree_args a;
        std::memcpy(&a, args, sizeof(a));
        if (a.depth < 0 || a.depth > 30 || a.iters < 0 || a.K < 1 || a.K > 4 || a.cutoff < 0 || a.cutoff > 20 ||
            (type == T_BINTREE && a.cutoff != 0))
            return GTAP_ERR_INVALID_ARG;
        struct { unsigned long long id; uint32_t level, depth, iters, kr; unsigned long long acc; } p{
            1ull, 0u, (uint32_t)a.depth, (uint32_t)a.iters,
            (uint32_t)a.K | ((a.route ? 1u : 0u) << 8) | ((uint32_t)a.cutoff << 16), 0ull};
        put(&p, sizeof(p));
        return GTAP_OK;
    }
    case T_TSORT: {
        if (nbytes != sizeof(gtap_cilksort_args)) return GTAP_ERR_INVALID_ARG;
        gtap_cilksort_args a;
        std::memcpy(&a, args, sizeof(a));
        if (a.sort_cutoff == 0) a.sort_cutoff = 64;
        if (a.merge_cutoff == 0) a.merge_cutoff = 256;
        if (a.n >= (1ull << 32) || a.sort_cutoff > 256 || a.merge_cutoff < 1 ||
            (a.n > 0 && (!a.src || !a.dst || !a.tmp)))
            return GTAP_ERR_INVALID_ARG;
        struct { uint32_t root, into, lo, hi; } p{root_index, 0u, 0u, (uint32_t)a.n};
        put(&p, sizeof(p));
        std::memcpy(d->env, &a, sizeof(a));
        return GTAP_OK;
    }
    case T_INTEGRATE_BLK: {
        if (nbytes != sizeof(gtap_integrate_args)) return GTAP_ERR_INVALID_ARG;
        gtap_integrate_args a;
        std::memcpy(&a, args, sizeof(a));
        if (!(a.eps > 0.0)) return GTAP_ERR_INVALID_ARG;
        double p[4] = {a.a, a.b, a.eps, 0.0};
        put(p, sizeof(p));
        return GTAP_OK;
    }
    case T_DTT: {
        if (nbytes != sizeof(gtap_fmm_dtt_args)) return GTAP_ERR_INVALID_ARG;
        gtap_fmm_dtt_args a;
        std::memcpy(&a, args, sizeof(a));
        fmm::DttEnv env;
        gtap_status st = fmm::dtt_env(a.plan, a.target, a.source, &env);
        if (st != GTAP_OK) return st;
        struct { uint32_t root, n; unsigned long long pr; } p{
            root_index, 1u, ((unsigned long long)(uint32_t)a.target << 32) | (uint32_t)a.source};
        put(&p, sizeof(p));
        std::memcpy(d->env, &env, sizeof(env));
        return GTAP_OK;
    }
    case T_MSORT: {
        if (nbytes != sizeof(gtap_mergesort_args)) return GTAP_ERR_INVALID_ARG;
        gtap_mergesort_args a;
        std::memcpy(&a, args, sizeof(a));
        if (a.leaf == 0) a.leaf = 4096;
        if (a.merge_cutoff == 0) a.merge_cutoff = 4096;
        if (a.leaf > 4096 || a.merge_cutoff < 256 || a.merge_cutoff > (1u << 20)) return GTAP_ERR_INVALID_ARG;
        if (a.n > 0 && (!a.src || !a.dst || (!a.tmp && a.n > a.leaf))) return GTAP_ERR_INVALID_ARG;
        struct { uint32_t root, into_tmp; unsigned long long lo, hi; } p{root_index, 0u, 0ull, a.n};
        put(&p, sizeof(p));
        std::memcpy(d->env, &a, sizeof(a));
        return GTAP_OK;
    }
    default:
        return GTAP_ERR_INVALID_ARG;
    }
}

gtap_status gtap_spawn_root(gtap_ctx* c, int type, const void* args, size_t args_bytes, int queue, uint64_t* out_handle) {
    if (!c || !args || type <= 0 || type >= T_MAX || !c->registered_type[type]) return GTAP_ERR_INVALID_ARG;
    if (queue < 0 || queue >= c->n_queues) return GTAP_ERR_INVALID_ARG;
    if (c->running) return GTAP_ERR_BUSY;
    if ((int)c->pending_roots.size() >= c->cfg.max_roots) return GTAP_ERR_INVALID_ARG;
    RootDesc d;
    const uint32_t idx = (uint32_t)c->pending_roots.size();
    gtap_status s = make_root(c, type, args, args_bytes, queue, idx, &d);
    if (s != GTAP_OK) return s;
    c->pending_roots.push_back(d);
    if (out_handle) *out_handle = idx;
    drop_graph(c);
    return GTAP_OK;
}

gtap_status gtap_clear_roots(gtap_ctx* c) {
    if (!c) return GTAP_ERR_INVALID_ARG;
    if (c->running) return GTAP_ERR_BUSY;
    c->pending_roots.clear();
    c->have_results = false;
    drop_graph(c);
    return GTAP_OK;
}

gtap_status gtap_set_timeout(gtap_ctx* c, uint64_t timeout_ns) {
    if (!c) return GTAP_ERR_INVALID_ARG;
    if (c->running) return GTAP_ERR_BUSY;
    c->cfg.timeout_ns = timeout_ns ? timeout_ns : 60ull * 1000000000ull;
    drop_graph(c);   // a captured run carries the old deadline
    return GTAP_OK;
}

struct LaunchPlan {
    KParams P;
    unsigned pset;
    size_t smem;
    int grid;
};

static gtap_status plan_and_enqueue(gtap_ctx* c, cudaStream_t s, LaunchPlan* lp, bool capturing = false,
                                    bool serving = false);

gtap_status gtap_run(gtap_ctx* c) {
    if (!c) return GTAP_ERR_INVALID_ARG;
    if (c->running || c->serving) return GTAP_ERR_BUSY;
    const uint32_t nroots = (uint32_t)c->pending_roots.size();
    if (nroots == 0) return GTAP_ERR_INVALID_ARG;
    if (c->graph_valid) {
        // replay the captured run (root upload + reset + persistent kernel)
        *c->host_abort = 0;
        cudaStream_t s = c->own_stream;
        cudaEventRecord(c->ev_start, s);
        if (cudaGraphLaunch(c->graph_exec, s) != cudaSuccess) { cudaGetLastError(); return GTAP_ERR_CUDA; }
        cudaEventRecord(c->ev_stop, s);
        c->running = true;
        c->have_results = false;
        c->run_stream = s;
        c->launched_roots = c->graph_roots;
        c->launched_workers = c->graph_workers;
        c->launched_grid = c->graph_grid;
        c->launched_frames = c->graph_frames;
        return GTAP_OK;
    }
    LaunchPlan lp;
    cudaStream_t s = c->stream;
    cudaEventRecord(c->ev_start, s);
    gtap_status st = plan_and_enqueue(c, s, &lp);
    if (st != GTAP_OK) return st;
    cudaEventRecord(c->ev_stop, s);
    c->running = true;
    c->have_results = false;
    c->run_stream = s;
    c->launched_roots = nroots;
    c->launched_workers = lp.P.n_workers;
    c->launched_grid = lp.grid;
    c->launched_frames = lp.P.n_frames;
    return GTAP_OK;
}

gtap_status gtap_capture_graph(gtap_ctx* c) {
    if (!c) return GTAP_ERR_INVALID_ARG;
    if (c->running) return GTAP_ERR_BUSY;
    if (c->pending_roots.empty()) return GTAP_ERR_INVALID_ARG;
    drop_graph(c);
    if (!c->own_stream && cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) return GTAP_ERR_CUDA;
    // make sure earlier work on the user stream is done before capturing the first replay's inputs
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return GTAP_ERR_CUDA;
    LaunchPlan lp;
    if (cudaStreamBeginCapture(c->own_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GTAP_ERR_CUDA;
    gtap_status st = plan_and_enqueue(c, c->own_stream, &lp, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->own_stream, &g);
    if (st != GTAP_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess || !g) { cudaGetLastError(); return GTAP_ERR_CUDA; }
    if (cudaGraphInstantiate(&c->graph_exec, g, 0) != cudaSuccess) { cudaGetLastError(); cudaGraphDestroy(g); return GTAP_ERR_CUDA; }
    c->graph = g;
    c->graph_valid = true;
    c->graph_roots = (uint32_t)c->pending_roots.size();
    c->graph_workers = lp.P.n_workers;
    c->graph_grid = lp.grid;
    c->graph_frames = lp.P.n_frames;
    return GTAP_OK;
}

static gtap_status plan_and_enqueue(gtap_ctx* c, cudaStream_t s, LaunchPlan* lp, bool capturing, bool serving) {
    // inside a capture the kernel-timing events become event-record nodes of the graph
    auto record = [&](cudaEvent_t ev) {
        if (capturing) cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
        else cudaEventRecord(ev, s);
    };
    const uint32_t nroots = serving ? 0u : (uint32_t)c->pending_roots.size();

    KParams P{};
    unsigned pset;
    int maxspawn;
    size_t smem;
    int grid = c->grid;
    uint32_t frame_bytes;
    if (c->mode == GTAP_MODE_THREAD) {
        pset = thread_kernel_pset(c->registered);
        maxspawn = thread_kernel_maxspawn(pset);
        frame_bytes = c->cfg.frame_bytes ? (uint32_t)c->cfg.frame_bytes : thread_record_bytes(pset);
        P.warp_smem = (uint32_t)(thread_warp_smem(maxspawn) + thread_prog_smem(pset));
        smem = (size_t)(c->threads_per_block / 32) * P.warp_smem;
        int occ = 0;
        {
            const cudaError_t oe = thread_kernel_occupancy(pset, c->cfg.scheduler, c->threads_per_block, smem, &occ);
            if (oe == cudaErrorInvalidValue) { cudaGetLastError(); return GTAP_ERR_INVALID_ARG; }   // no such instantiation
            if (oe != cudaSuccess) return GTAP_ERR_CUDA;
        }
        if (occ < 1) return GTAP_ERR_INVALID_ARG;
        grid = std::min(c->grid, occ * c->sm_count);
        P.n_workers = (uint32_t)(grid * (c->threads_per_block / 32));
    } else {
        pset = block_kernel_pset(c->registered);
        maxspawn = block_kernel_maxspawn(pset, c->threads_per_block);
        frame_bytes = block_record_bytes(pset, c->threads_per_block);
        smem = (size_t)block_rt_smem(maxspawn) + block_prog_smem(pset, c->threads_per_block);
        int occ = 0;
        {
            const cudaError_t oe = block_kernel_occupancy(pset, c->threads_per_block, smem, &occ);
            if (oe == cudaErrorInvalidValue) { cudaGetLastError(); return GTAP_ERR_INVALID_ARG; }   // no such instantiation
            if (oe != cudaSuccess) return GTAP_ERR_CUDA;
        }
        if (occ < 1) return GTAP_ERR_INVALID_ARG;
        grid = std::min(c->grid, occ * c->sm_count);
        P.n_workers = (uint32_t)grid;
    }
    const uint64_t n_frames = std::min<uint64_t>(c->pool_bytes / frame_bytes, 0x7FFFFFF0ull);
    if (n_frames < nroots) return GTAP_ERR_POOL_EXHAUSTED;
    // roots per worker queue must fit in a ring
    if ((nroots + P.n_workers - 1) / P.n_workers > c->ring_cap) return GTAP_ERR_DEQUE_OVERFLOW;

    P.frames = c->frames;
    P.n_frames = n_frames;
    P.frame_bytes = frame_bytes;
    P.n_queues = (uint32_t)c->n_queues;
    P.ring_mask = c->ring_cap - 1;
    P.rings = c->rings;
    P.qs = c->qs;
    P.cq_seq = c->cq_seq;
    P.cq_ids = c->cq_ids;
    P.ncq_mask = c->ncq - 1;
    P.ctl = c->ctl;
    P.roots = c->roots;
    P.root_desc = c->root_desc;
    P.n_roots = nroots;
    P.maxspawn = (uint32_t)maxspawn;
    P.stats = c->stats;
    P.host_abort = c->host_abort_dev;
    P.timeout_ns = c->cfg.timeout_ns;
    P.seed = c->cfg.seed;
    P.steal_policy = c->cfg.steal_policy;
    P.idle_backoff_ns = c->cfg.idle_backoff_ns;
    P.scratch = c->blocks;
    P.scratch_bytes = c->blocks_bytes;
    P.sq_seq = c->sq_seq;
    P.sq_ids = c->sq_ids;
    P.sq_mask = c->sq_mask;
    P.lq_seq = c->lq_seq;
    P.lq_ids = c->lq_ids;
    P.lq_mask = c->lq_mask;
    P.fstate = c->fstate;
    P.flog = c->flog;
    P.flogn = c->flogn;
    P.gq = c->gq;
    P.gq_mask = c->gq_cap ? c->gq_cap - 1 : 0;
    if (c->flogn) cudaMemsetAsync(c->flogn, 0, c->max_frames * sizeof(unsigned), c->stream);

    *c->host_abort = 0;
    if (nroots > 0) {
        std::memcpy(c->root_desc_pinned, c->pending_roots.data(), nroots * sizeof(RootDesc));
        if (cudaMemcpyAsync(c->root_desc, c->root_desc_pinned, nroots * sizeof(RootDesc), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return GTAP_ERR_CUDA;
    }
    if (launch_reset(P, 1, s) != cudaSuccess) return GTAP_ERR_CUDA;
    if (serving) {
        // the root table becomes a ring of request slots for the whole session
        P.serving = 1;
        P.n_roots = (uint32_t)c->cfg.max_roots;
        P.inbox = c->inbox_dev;
        P.inbox_cap = (uint32_t)c->cfg.max_roots;
        P.outbox = c->outbox_dev;
        P.outbox_cap = (uint32_t)c->cfg.max_roots;
        P.hflags = c->hflags_dev;
        P.host_abort = &c->hflags_dev->abort;
        P.admit_reserve = std::max<uint64_t>(P.n_frames / 64, 4096);
        // every request slot starts free (all bytes 0xFF: done == kRootSlotFree)
        if (cudaMemsetAsync(c->roots, 0xFF, (size_t)c->cfg.max_roots * sizeof(RootEntry), s) != cudaSuccess)
            return GTAP_ERR_CUDA;
    }
    record(c->ev_k0);
    cudaError_t e = (c->mode == GTAP_MODE_THREAD)
                        ? launch_thread_kernel(pset, c->cfg.scheduler, P, grid, c->threads_per_block, smem, s)
                        : launch_block_kernel(pset, c->threads_per_block, P, grid, smem, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GTAP_ERR_CUDA;
    }
    record(c->ev_k1);
    lp->P = P;
    lp->pset = pset;
    lp->smem = smem;
    lp->grid = grid;
    return GTAP_OK;
}

gtap_status gtap_wait(gtap_ctx* c, uint64_t timeout_ms) {
    if (!c) return GTAP_ERR_INVALID_ARG;
    if (!c->running) return c->have_results ? (gtap_status)c->last_err.code : GTAP_ERR_INVALID_ARG;
    if (timeout_ms == 0) timeout_ms = c->cfg.timeout_ns / 1000000ull + 5000ull;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    bool timed_out = false;
    while (true) {
        cudaError_t q = cudaEventQuery(c->ev_stop);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) { c->running = false; return GTAP_ERR_CUDA; }
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(clk::now() - t0).count();
        if (!timed_out && (uint64_t)ms > timeout_ms) {
            // ask the kernel to drain through the mapped abort word, then keep waiting (bounded)
            *reinterpret_cast<volatile int*>(c->host_abort) = 1;
            timed_out = true;
        }
        if (timed_out && (uint64_t)ms > timeout_ms + 10000ull) { return GTAP_ERR_TIMEOUT; }
        std::this_thread::sleep_for(std::chrono::microseconds(ms < 2 ? 20 : 200));
    }
    c->running = false;
    float kms = 0.f, rms = 0.f;
    cudaEventElapsedTime(&kms, c->ev_k0, c->ev_k1);
    cudaEventElapsedTime(&rms, c->ev_start, c->ev_stop);
    cudaStream_t s = c->run_stream;
    if (cudaMemcpyAsync(c->ctl_pinned, c->ctl, sizeof(DevControl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(c->roots_pinned, c->roots, c->launched_roots * sizeof(RootEntry), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(c->stats_pinned, c->stats, c->launched_workers * sizeof(WorkerStats), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GTAP_ERR_CUDA;
    gtap_stats st{};
    for (uint32_t w = 0; w < c->launched_workers; ++w) {
        const WorkerStats& x = c->stats_pinned[w];
        st.tasks_executed += x.tasks;
        st.steps += x.steps;
        st.pops += x.pops;
        st.popped += x.popped;
        st.steal_attempts += x.steal_attempts;
        st.steals += x.steals;
        st.stolen += x.stolen;
        st.idle_iterations += x.idle;
        st.pushes += x.pushes;
        st.pushed += x.pushed;
        st.tasks_created += x.spawned;
        // thread mode: pop, steal, execute, retain/push, idle; block mode: acquire (pop or
        // steal), -, body, post-step, idle
        st.cycles_pop += x.pad[0]; st.cycles_steal += x.pad[1]; st.cycles_exec += x.pad[2];
        st.cycles_push += x.pad[3]; st.cycles_idle += x.pad[4];
    }
    st.tasks_created += c->launched_roots;
    st.frames_high_water = std::min<uint64_t>(c->ctl_pinned->bump.v, c->launched_frames);
    st.scratch_used = c->ctl_pinned->scratch_top.v * kScratchBlock;
    st.n_workers = (int)c->launched_workers;
    st.grid_blocks = c->launched_grid;
    st.threads_per_block = c->threads_per_block;
    st.kernel_ms = kms;
    st.run_ms = rms;
    c->last_stats = st;
    c->last_err.code = c->ctl_pinned->err.code;
    c->last_err.task_type = c->ctl_pinned->err.task_type;
    c->last_err.worker = c->ctl_pinned->err.worker;
    c->last_err.detail = c->ctl_pinned->err.detail;
    c->have_results = true;
    if (timed_out && c->last_err.code == 0) c->last_err.code = GTAP_ERR_TIMEOUT;
    return (gtap_status)c->last_err.code;
}

gtap_status gtap_serve_start(gtap_ctx* c) {
    if (!c || c->mode != GTAP_MODE_THREAD || c->registered == 0) return GTAP_ERR_INVALID_ARG;
    if (c->running || c->serving) return GTAP_ERR_BUSY;
    const size_t cap = (size_t)c->cfg.max_roots;
    if (!c->inbox) {
        if (cudaHostAlloc(reinterpret_cast<void**>(&c->inbox), cap * sizeof(InboxSlot), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void**>(&c->outbox), cap * sizeof(OutboxEntry), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void**>(&c->hflags), sizeof(HostFlags), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->inbox_dev), c->inbox, 0) != cudaSuccess ||
            cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->outbox_dev), c->outbox, 0) != cudaSuccess ||
            cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->hflags_dev), c->hflags, 0) != cudaSuccess) {
            cudaGetLastError();
            return GTAP_ERR_NO_MEMORY;
        }
    }
    std::memset(c->inbox, 0, cap * sizeof(InboxSlot));
    std::memset(c->outbox, 0, cap * sizeof(OutboxEntry));
    std::memset(c->hflags, 0, sizeof(HostFlags));
    c->submitted = 0;
    if (!c->own_stream && cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) return GTAP_ERR_CUDA;
    LaunchPlan lp;
    cudaStream_t s = c->own_stream;
    cudaEventRecord(c->ev_start, s);
    gtap_status st = plan_and_enqueue(c, s, &lp, false, true);
    if (st != GTAP_OK) return st;
    cudaEventRecord(c->ev_stop, s);
    c->serving = true;
    c->running = true;
    c->have_results = false;
    c->run_stream = s;
    c->launched_roots = 0;
    c->launched_workers = lp.P.n_workers;
    c->launched_grid = lp.grid;
    c->launched_frames = lp.P.n_frames;
    return GTAP_OK;
}

gtap_status gtap_submit(gtap_ctx* c, int type, const void* args, size_t args_bytes, int queue, uint64_t* out_req) {
    if (!c || !c->serving || !args || type <= 0 || type >= T_MAX || !c->registered_type[type]) return GTAP_ERR_INVALID_ARG;
    if (queue < 0 || queue >= c->n_queues) return GTAP_ERR_INVALID_ARG;
    const uint64_t cap = (uint64_t)c->cfg.max_roots;
    volatile HostFlags* hf = c->hflags;
    if (c->submitted - hf->inbox_consumed >= cap) return GTAP_ERR_BUSY;
    RootDesc d;
    gtap_status st = make_root(c, type, args, args_bytes, queue, 0, &d);
    if (st != GTAP_OK) return st;
    InboxSlot* slot = c->inbox + (c->submitted % cap);
    slot->type = d.type;
    slot->queue = d.queue;
    std::memcpy(slot->payload, d.payload, sizeof(slot->payload));
    std::memcpy(slot->env, d.env, sizeof(slot->env));
    std::atomic_thread_fence(std::memory_order_release);
    reinterpret_cast<volatile InboxSlot*>(slot)->seq = c->submitted + 1;
    if (out_req) *out_req = c->submitted;
    ++c->submitted;
    return GTAP_OK;
}

gtap_status gtap_poll(gtap_ctx* c, gtap_completion* out, int max, int* n) {
    if (!c || !n || max < 0 || (max > 0 && !out) || !c->hflags) return GTAP_ERR_INVALID_ARG;
    const uint64_t cap = (uint64_t)c->cfg.max_roots;
    volatile HostFlags* hf = c->hflags;
    uint64_t oc = hf->out_consumed;
    int k = 0;
    while (k < max) {
        volatile OutboxEntry* e = c->outbox + (oc % cap);
        if (e->seq != oc + 1) break;
        std::atomic_thread_fence(std::memory_order_acquire);
        out[k].req = e->req;
        out[k].result[0] = e->result[0];
        out[k].result[1] = e->result[1];
        out[k].status = e->status;
        out[k].pad = 0;
        ++k;
        ++oc;
    }
    std::atomic_thread_fence(std::memory_order_release);
    hf->out_consumed = oc;
    *n = k;
    return (gtap_status)hf->dev_error;
}

gtap_status gtap_serve_progress(gtap_ctx* c, uint64_t* out, int n) {
    if (!c || !out || n < 0 || !c->hflags) return GTAP_ERR_INVALID_ARG;
    volatile HostFlags* hf = c->hflags;
    const uint64_t v[3] = {c->submitted, hf->inbox_consumed, hf->out_consumed};
    for (int i = 0; i < n && i < 3; ++i) out[i] = v[i];
    return GTAP_OK;
}

gtap_status gtap_serve_stop(gtap_ctx* c, uint64_t timeout_ms) {
    if (!c || !c->serving) return GTAP_ERR_INVALID_ARG;
    std::atomic_thread_fence(std::memory_order_release);
    reinterpret_cast<volatile HostFlags*>(c->hflags)->shutdown = c->submitted + 1;
    gtap_status st = gtap_wait(c, timeout_ms);
    c->serving = false;
    return st;
}

gtap_status gtap_read_result(gtap_ctx* c, uint64_t handle, void* out, size_t bytes) {
    if (!c || !out || bytes > 16) return GTAP_ERR_INVALID_ARG;
    if (!c->have_results) return GTAP_ERR_NOT_READY;
    if (handle >= c->launched_roots) return GTAP_ERR_INVALID_ARG;
    const RootEntry& r = c->roots_pinned[handle];
    if (!r.done) return GTAP_ERR_NOT_READY;
    std::memcpy(out, r.result, bytes);
    return GTAP_OK;
}

gtap_status gtap_get_stats(gtap_ctx* c, gtap_stats* out) {
    if (!c || !out) return GTAP_ERR_INVALID_ARG;
    *out = c->last_stats;
    return GTAP_OK;
}

gtap_status gtap_last_error(gtap_ctx* c, gtap_error_info* out) {
    if (!c || !out) return GTAP_ERR_INVALID_ARG;
    *out = c->last_err;
    return GTAP_OK;
}

gtap_status gtap_debug_snapshot(gtap_ctx* c, uint64_t* out, int n) {
    if (!c || !out || n < 0) return GTAP_ERR_INVALID_ARG;
    if (c->running) return GTAP_ERR_BUSY;
    const size_t qn = (size_t)c->n_workers_max * c->n_queues;
    std::vector<QState> qs(qn);
    DevControl ctl;
    if (cudaMemcpy(qs.data(), c->qs, qn * sizeof(QState), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&ctl, c->ctl, sizeof(ctl), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GTAP_ERR_CUDA;
    uint64_t v[9] = {ctl.roots_remaining.v, ctl.bump.v, ctl.cq_enq.v, ctl.cq_deq.v, 0, 0, 0, 0, ctl.abort_flag.v};
    for (const QState& q : qs) {
        if (q.count > 0) { v[4] += (uint64_t)q.count; ++v[5]; v[7] = std::max<uint64_t>(v[7], (uint64_t)q.count); }
        if (q.lock) ++v[6];
    }
    for (int i = 0; i < n && i < 9; ++i) out[i] = v[i];
    return GTAP_OK;
}

gtap_status gtap_debug_record_log(gtap_ctx* c, uint32_t id, uint64_t* out) {
    if (!c || !out || !c->flog || id >= c->max_frames) return GTAP_ERR_INVALID_ARG;
    if (c->running) return GTAP_ERR_BUSY;
    unsigned n = 0;
    if (cudaMemcpy(&n, c->flogn + id, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(out + 1, c->flog + (size_t)id * 8, 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GTAP_ERR_CUDA;
    out[0] = n;
    return GTAP_OK;
}

gtap_status gtap_finalize(gtap_ctx* c) {
    if (!c) return GTAP_ERR_INVALID_ARG;
    if (c->running) {
        gtap_status s = gtap_wait(c, 0);
        if (s == GTAP_ERR_TIMEOUT && c->running) return GTAP_ERR_BUSY;
    }
    return free_all(c);
}

}  // extern "C"
