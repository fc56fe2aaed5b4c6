// Device runtime: memory-ordering primitives, task-record pool, deques and the
// persistent scheduler loops (thread mode and block mode).
//
// Sec. 5.1 of the paper describes the design this follows: one persistent
// kernel, per-warp (thread mode) or per-block (block mode) ring-buffer deques
// whose `head` and `count` live in global memory and are accessed through L2
// while the owner's `tail` lives in shared memory; batched pop/steal claims by
// CAS on `count` (Algorithm 2); one fence and one `count` increment per push
// batch; suspension at a join with a waiting-child counter whose last
// decrement re-enqueues the parent (Sec. 5.1.2).
#pragma once
#include <cstdint>
#include "gtap_internal.h"
#include "gtap.h"

namespace gtap {

// ---------------------------------------------------------------------------
// Memory primitives.  Every cross-SM word is accessed through L2 (.cg loads,
// atomics); publication uses release/acquire at GPU scope.
__device__ __forceinline__ uint32_t ld_cg32(const void* p) { return __ldcg(reinterpret_cast<const unsigned int*>(p)); }
__device__ __forceinline__ int ld_cg_i32(const int* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ld_cg64(const void* p) {
    return __ldcg(reinterpret_cast<const unsigned long long*>(p));
}
__device__ __forceinline__ void st_cg32(void* p, uint32_t v) { __stcg(reinterpret_cast<unsigned int*>(p), v); }
__device__ __forceinline__ void st_cg64(void* p, unsigned long long v) {
    __stcg(reinterpret_cast<unsigned long long*>(p), v);
}

__device__ __forceinline__ uint32_t atom_add_acqrel_u32(void* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ int atom_cas_acq_i32(int* p, int cmp, int val) {
    int old;
    asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "l"(p), "r"(cmp), "r"(val) : "memory");
    return old;
}
__device__ __forceinline__ unsigned long long atom_cas_acq_u64(unsigned long long* p, unsigned long long cmp,
                                                               unsigned long long val) {
    unsigned long long old;
    asm volatile("atom.acquire.gpu.global.cas.b64 %0, [%1], %2, %3;" : "=l"(old) : "l"(p), "l"(cmp), "l"(val) : "memory");
    return old;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned int* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Copy a trivially copyable object through L2 in 16/8/4-byte pieces.
template <class T>
__device__ __forceinline__ T ld_obj(const void* src) {
    static_assert(sizeof(T) % 4 == 0, "record fields must be 4-byte multiples");
    T out;
    if constexpr (sizeof(T) % 16 == 0) {
        uint4 tmp[sizeof(T) / 16];
#pragma unroll
        for (int i = 0; i < (int)(sizeof(T) / 16); ++i) tmp[i] = __ldcg(reinterpret_cast<const uint4*>(src) + i);
        memcpy(&out, tmp, sizeof(T));
    } else if constexpr (sizeof(T) % 8 == 0) {
        uint2 tmp[sizeof(T) / 8];
#pragma unroll
        for (int i = 0; i < (int)(sizeof(T) / 8); ++i) tmp[i] = __ldcg(reinterpret_cast<const uint2*>(src) + i);
        memcpy(&out, tmp, sizeof(T));
    } else {
        unsigned int tmp[sizeof(T) / 4];
#pragma unroll
        for (int i = 0; i < (int)(sizeof(T) / 4); ++i) tmp[i] = __ldcg(reinterpret_cast<const unsigned int*>(src) + i);
        memcpy(&out, tmp, sizeof(T));
    }
    return out;
}
// The same through the read-only (non-coherent) path: for data that no thread
// writes while the kernel runs (root environments of a batch run).
template <class T>
__device__ __forceinline__ T ld_obj_ro(const void* src) {
    static_assert(sizeof(T) % 8 == 0, "read-only objects are copied in 8-byte pieces");
    T out;
    if constexpr (sizeof(T) % 16 == 0) {
        uint4 tmp[sizeof(T) / 16];
#pragma unroll
        for (int i = 0; i < (int)(sizeof(T) / 16); ++i) tmp[i] = __ldg(reinterpret_cast<const uint4*>(src) + i);
        memcpy(&out, tmp, sizeof(T));
    } else {
        uint2 tmp[sizeof(T) / 8];
#pragma unroll
        for (int i = 0; i < (int)(sizeof(T) / 8); ++i) tmp[i] = __ldg(reinterpret_cast<const uint2*>(src) + i);
        memcpy(&out, tmp, sizeof(T));
    }
    return out;
}

template <class T>
__device__ __forceinline__ void st_obj(void* dst, const T& v) {
    static_assert(sizeof(T) % 4 == 0, "record fields must be 4-byte multiples");
    if constexpr (sizeof(T) % 16 == 0) {
        uint4 tmp[sizeof(T) / 16];
        memcpy(tmp, &v, sizeof(T));
#pragma unroll
        for (int i = 0; i < (int)(sizeof(T) / 16); ++i) __stcg(reinterpret_cast<uint4*>(dst) + i, tmp[i]);
    } else if constexpr (sizeof(T) % 8 == 0) {
        uint2 tmp[sizeof(T) / 8];
        memcpy(tmp, &v, sizeof(T));
#pragma unroll
        for (int i = 0; i < (int)(sizeof(T) / 8); ++i) __stcg(reinterpret_cast<uint2*>(dst) + i, tmp[i]);
    } else {
        unsigned int tmp[sizeof(T) / 4];
        memcpy(tmp, &v, sizeof(T));
#pragma unroll
        for (int i = 0; i < (int)(sizeof(T) / 4); ++i) __stcg(reinterpret_cast<unsigned int*>(dst) + i, tmp[i]);
    }
}

__device__ __forceinline__ char* frame_ptr(const KParams& P, uint32_t id) {
    return P.frames + (uint64_t)id * P.frame_bytes;
}

// First error wins; every worker then drains (Sec. 4: structured error report).
static __device__ __noinline__ void raise_error(const KParams& P, int code, int task_type, int worker, unsigned long long detail) {
    if (atomicCAS(&P.ctl->err.code, 0, code) == 0) {
        P.ctl->err.task_type = task_type;
        P.ctl->err.worker = worker;
        P.ctl->err.detail = detail;
    }
    __threadfence();
    atomicExch(reinterpret_cast<unsigned long long*>(&P.ctl->abort_flag.v), 1ull);
    if (P.serving && P.hflags != nullptr) {
        // a served session reports the failure through mapped memory, where the host polls
        volatile int* e = &P.hflags->dev_error;
        if (*e == 0) *e = code;
        __threadfence_system();
    }
}

// Debug event log: code:4 | lane:5 | worker:15 | iteration:24 | aux:16.
// The debug paths below run only in debug contexts; their bodies are kept out
// of line so that the scheduler loops' hot code stays compact.
static __device__ __noinline__ void dbg_log_record(const KParams& P, uint32_t id, unsigned code, int worker,
                                                   uint32_t iter, unsigned aux) {
    if (id >= P.n_frames) return;
    unsigned k = atomicAdd(&P.flogn[id], 1u);
    unsigned long long ev = ((unsigned long long)code << 60) | ((unsigned long long)(threadIdx.x & 31) << 55) |
                            ((unsigned long long)(worker & 0x7FFF) << 40) | ((unsigned long long)(iter & 0xFFFFFF) << 16) |
                            (aux & 0xFFFF);
    P.flog[(size_t)id * 8 + (k & 7)] = ev;
}
__device__ __forceinline__ void dbg_log(const KParams& P, uint32_t id, unsigned code, int worker, uint32_t iter,
                                        unsigned aux) {
    if (P.flog != nullptr) dbg_log_record(P, id, code, worker, iter, aux);
}

// Debug checks on record ownership (only when P.fstate is set).
static __device__ __noinline__ void dbg_transition_check(const KParams& P, uint32_t id, unsigned from, unsigned to,
                                                         unsigned long long fault, int type, int worker) {
    if (id >= P.n_frames) { raise_error(P, GTAP_ERR_TASK_FAILED, type, worker, (DBG_BAD_ID << 32) | id); return; }
    unsigned old = atomicCAS(&P.fstate[id], from, to);
    if (old != from) raise_error(P, GTAP_ERR_TASK_FAILED, type, worker, (fault << 32) | id);
}
__device__ __forceinline__ void dbg_transition(const KParams& P, uint32_t id, unsigned from, unsigned to,
                                               unsigned long long fault, int type, int worker) {
    if (P.fstate != nullptr) dbg_transition_check(P, id, from, to, fault, type, worker);
}
// A task ID taken from a ring slot: the slot is cleared so that a second take of it is caught.
static __device__ __noinline__ void dbg_take_slot(const KParams& P, uint32_t* slot, uint32_t tid, int code, int worker) {
    uint32_t was = atomicExch(slot, kNoTask);
    if (was != tid || tid == kNoTask) raise_error(P, GTAP_ERR_TASK_FAILED, code, worker, (DBG_BAD_ID << 32) | was);
}
// A task about to run must be queued (3); it becomes running (2).
static __device__ __noinline__ void dbg_exec_check(const KParams& P, uint32_t tid, int src, int worker) {
    unsigned old = (tid < P.n_frames) ? atomicCAS(&P.fstate[tid], 3u, 2u) : 99u;
    if (old != 3u) raise_error(P, GTAP_ERR_TASK_FAILED, (int)(old * 16 + src), worker, (DBG_EXEC_NOT_ALLOCATED << 32) | tid);
}
// A record is queued only from "allocated" (1), or from "running" (2) by itself; returns true
// when the running task staged itself.
static __device__ __noinline__ bool dbg_stage_check(const KParams& P, uint32_t id, uint32_t self, uint32_t parent,
                                                    int worker) {
    unsigned old = atomicCAS(&P.fstate[id], 1u, 3u);
    if (old == 1u) return false;
    if (id == self && old == 2u && atomicCAS(&P.fstate[id], 2u, 3u) == 2u) return true;
    raise_error(P, GTAP_ERR_TASK_FAILED, (int)(200 + old * 16 + (id == self ? 1 : 0) + (id == parent ? 2 : 0)), worker,
                (5ull << 32) | id);
    return false;
}

__device__ __forceinline__ bool abort_requested(const KParams& P, bool check_host) {
    if (ld_cg64(&P.ctl->abort_flag.v) != 0) return true;
    // the host word lives in mapped host memory (a slow read): checked less often
    if (check_host && P.host_abort != nullptr && *P.host_abort != 0) {
        atomicExch(reinterpret_cast<unsigned long long*>(&P.ctl->abort_flag.v), 1ull);
        return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// Scratch blocks (lane-level).  Programs that need variable-size buffers during
// a run (k-clique candidate sets) take kScratchBlock-byte blocks: recycled
// blocks come from a bounded MPMC queue with fetch-and-add tickets and a
// completed-free counter (the frame pool's chunk-queue protocol, one block per
// slot), fresh ones from a bump counter.  Buffers larger than one block take
// consecutive fresh blocks and are not recycled.
// A bounded MPMC queue of free ids (the frame pool's chunk-queue protocol, one id per slot).
struct FreeQ {
    unsigned long long* seq;
    uint32_t* ids;
    uint64_t mask;
    unsigned long long *enq, *deq, *avail;
};
__device__ __forceinline__ FreeQ small_free_q(const KParams& P) {
    return FreeQ{P.sq_seq, P.sq_ids, P.sq_mask, &P.ctl->sc_enq.v, &P.ctl->sc_deq.v, &P.ctl->sc_avail.v};
}
__device__ __forceinline__ FreeQ large_free_q(const KParams& P) {
    return FreeQ{P.lq_seq, P.lq_ids, P.lq_mask, &P.ctl->lc_enq.v, &P.ctl->lc_deq.v, &P.ctl->lc_avail.v};
}

// Take a free id: >= 0 the id, -1 none free, -2 a wait ran out (error raised).
__device__ __forceinline__ long long freeq_take(const KParams& P, const FreeQ& q, int type, int worker) {
    const long long a = (long long)atomicAdd(q.avail, ~0ull);   // reserve one completed free
    if (a <= 0) { atomicAdd(q.avail, 1ull); return -1; }
    const unsigned long long d = atomicAdd(q.deq, 1ull);
    for (int it = 0; it < (1 << 20); ++it) {
        if (ld_acquire_u64(&q.seq[d & q.mask]) == d + 1) {
            const uint32_t id = __ldcg(&q.ids[d & q.mask]);
            st_release_u64(&q.seq[d & q.mask], d + q.mask + 1);
            return (long long)id;
        }
        __nanosleep(64);
    }
    raise_error(P, GTAP_ERR_TASK_FAILED, type, worker, d);
    return -2;
}

__device__ __forceinline__ void freeq_give(const KParams& P, const FreeQ& q, uint32_t id, int type, int worker) {
    const unsigned long long t = atomicAdd(q.enq, 1ull);
    for (int it = 0; it < (1 << 20); ++it) {
        if (ld_acquire_u64(&q.seq[t & q.mask]) == t) {
            __stcg(&q.ids[t & q.mask], id);
            __threadfence();
            st_release_u64(&q.seq[t & q.mask], t + 1);
            atomicAdd(q.avail, 1ull);
            return;
        }
        __nanosleep(64);
    }
    raise_error(P, GTAP_ERR_TASK_FAILED, type, worker, t);
}

// Scratch buffers.  kind: 1 = one recycled block (<= kScratchBlock bytes),
// 2 = a recycled large chunk (<= kScratchLargeBlocks blocks), 0 = larger,
// consecutive fresh blocks that are not recycled.  Returns null after raising
// GTAP_ERR_TASK_FAILED when the arena is exhausted.
__device__ __forceinline__ char* scratch_alloc_kind(const KParams& P, uint64_t bytes, int* kind, int type, int worker) {
    const uint64_t nblocks = P.scratch_bytes / kScratchBlock;
    uint64_t k = (bytes + kScratchBlock - 1) / kScratchBlock;
    *kind = 0;
    if (k <= 1) {
        *kind = 1;
        k = 1;
        const long long id = freeq_take(P, small_free_q(P), type, worker);
        if (id == -2) return nullptr;
        if (id >= 0) return P.scratch + (uint64_t)id * kScratchBlock;
    } else if (k <= kScratchLargeBlocks && P.lq_seq != nullptr) {
        *kind = 2;
        k = kScratchLargeBlocks;
        const long long id = freeq_take(P, large_free_q(P), type, worker);
        if (id == -2) return nullptr;
        if (id >= 0) return P.scratch + (uint64_t)id * kScratchBlock;
    }
    const unsigned long long b = atomicAdd(&P.ctl->scratch_top.v, (unsigned long long)k);
    if (b + k > nblocks) { raise_error(P, GTAP_ERR_TASK_FAILED, type, worker, (b + k) * kScratchBlock); return nullptr; }
    return P.scratch + b * kScratchBlock;
}

__device__ __forceinline__ char* scratch_alloc(const KParams& P, uint64_t bytes, bool* pooled, int type, int worker) {
    // one recycled block, or consecutive fresh blocks that are not recycled
    if (bytes <= kScratchBlock) {
        int kind;
        char* p = scratch_alloc_kind(P, bytes, &kind, type, worker);
        *pooled = true;
        return p;
    }
    *pooled = false;
    const uint64_t nblocks = P.scratch_bytes / kScratchBlock;
    const uint64_t k = (bytes + kScratchBlock - 1) / kScratchBlock;
    const unsigned long long b = atomicAdd(&P.ctl->scratch_top.v, (unsigned long long)k);
    if (b + k > nblocks) { raise_error(P, GTAP_ERR_TASK_FAILED, type, worker, (b + k) * kScratchBlock); return nullptr; }
    return P.scratch + b * kScratchBlock;
}

__device__ __forceinline__ uint32_t scratch_block_id(const KParams& P, const void* p) {
    return (uint32_t)((reinterpret_cast<const char*>(p) - P.scratch) / kScratchBlock);
}
__device__ __forceinline__ void scratch_free(const KParams& P, const void* p, int type, int worker) {
    freeq_give(P, small_free_q(P), scratch_block_id(P, p), type, worker);
}
// Release a buffer by the kind scratch_alloc_kind returned (kind 0 is never recycled).
__device__ __forceinline__ void scratch_free_kind(const KParams& P, const void* p, int kind, int type, int worker) {
    if (kind == 1) freeq_give(P, small_free_q(P), scratch_block_id(P, p), type, worker);
    else if (kind == 2) freeq_give(P, large_free_q(P), scratch_block_id(P, p), type, worker);
}

// ---------------------------------------------------------------------------
// Frame pool.  Free IDs are cached per worker in shared memory; surplus is
// moved to / from a global bounded MPMC queue of 32-ID chunks (sequence-number
// slots, after Vyukov's bounded queue); never-used IDs come from a bump
// pointer.  All of it is warp-collective (called by one full warp).

// Chunk queue protocol.  Tickets come from fetch-and-add on cq_enq / cq_deq,
// so no operation retries under contention.  cq_avail counts the chunks whose
// enqueue has completed: a dequeuer first reserves chunks from it (undoing an
// over-reservation), so every dequeue ticket it then takes belongs to an
// enqueue already in progress, and the wait for that slot's sequence number
// is short and bounded.  The queue has a slot for every chunk the pool can
// hold, so an enqueue ticket's slot is free once its previous occupant's
// dequeue finishes.

// Push k chunks (k * 32 IDs from src[0 .. 32k)) to the global queue (warp-collective).
__device__ __forceinline__ bool cq_push_many(const KParams& P, const uint32_t* src, int k) {
    const int lane = threadIdx.x & 31;
    unsigned long long t0 = 0;
    if (lane == 0) t0 = atomicAdd(&P.ctl->cq_enq.v, (unsigned long long)k);
    t0 = __shfl_sync(0xffffffffu, t0, 0);
    int ok = 1;
    for (int j = 0; j < k; ++j) {
        const unsigned long long slot = t0 + (unsigned long long)j;
        if (lane == 0) {
            int ready = 0;
            for (int it = 0; it < (1 << 20); ++it) {
                if (ld_acquire_u64(&P.cq_seq[slot & P.ncq_mask]) == slot) { ready = 1; break; }
                __nanosleep(64);
            }
            if (!ready) { raise_error(P, GTAP_ERR_TASK_FAILED, -1, -1, slot); ok = 0; }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) return false;
        __stcg(&P.cq_ids[(slot & P.ncq_mask) * kChunk + lane], src[j * kChunk + lane]);
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_u64(&P.cq_seq[slot & P.ncq_mask], slot + 1);
    }
    __syncwarp();
    if (lane == 0) { __threadfence(); atomicAdd(&P.ctl->cq_avail.v, (unsigned long long)k); }
    return true;
}

// Pop up to k chunks into dst[0 .. 32 * got) (warp-collective); returns got.
__device__ __forceinline__ int cq_pop_many(const KParams& P, uint32_t* dst, int k) {
    const int lane = threadIdx.x & 31;
    int got = 0;
    unsigned long long d0 = 0;
    if (lane == 0) {
        const long long a = (long long)atomicAdd(&P.ctl->cq_avail.v, (unsigned long long)(-(long long)k));
        got = (int)max(0ll, min((long long)k, a));
        if (got < k) atomicAdd(&P.ctl->cq_avail.v, (unsigned long long)(k - got));
        if (got > 0) d0 = atomicAdd(&P.ctl->cq_deq.v, (unsigned long long)got);
    }
    got = __shfl_sync(0xffffffffu, got, 0);
    d0 = __shfl_sync(0xffffffffu, d0, 0);
    for (int j = 0; j < got; ++j) {
        const unsigned long long slot = d0 + (unsigned long long)j;
        int ready = 1;
        if (lane == 0) {
            ready = 0;
            for (int it = 0; it < (1 << 20); ++it) {
                if (ld_acquire_u64(&P.cq_seq[slot & P.ncq_mask]) == slot + 1) { ready = 1; break; }
                __nanosleep(64);
            }
            if (!ready) raise_error(P, GTAP_ERR_TASK_FAILED, -1, -1, slot);
        }
        ready = __shfl_sync(0xffffffffu, ready, 0);
        if (!ready) return j;
        dst[j * kChunk + lane] = __ldcg(&P.cq_ids[(slot & P.ncq_mask) * kChunk + lane]);
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_u64(&P.cq_seq[slot & P.ncq_mask], slot + P.ncq_mask + 1);
    }
    __syncwarp();
    return got;
}

// Bring the local free stack up to `need` IDs (warp-collective).  Returns the
// new top; less than `need` only when the pool is exhausted.
__device__ __forceinline__ int pool_refill(const KParams& P, uint32_t* fstack, int ftop, int need) {
    const int lane = threadIdx.x & 31;
    if (ftop >= need) return ftop;
    const int k = (need - ftop + kChunk - 1) / kChunk;
    const int got = cq_pop_many(P, fstack + ftop, k);
    ftop += got * kChunk;
    if (got < k) {
        const int want = (k - got) * kChunk;
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(&P.ctl->bump.v, (unsigned long long)want);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b < P.n_frames) {
            const int avail = (int)min((unsigned long long)want, P.n_frames - b);
            for (int i = lane; i < avail; i += 32) fstack[ftop + i] = (uint32_t)(b + i);
            ftop += avail;
        }
    }
    __syncwarp();
    return ftop;
}

// Move whole chunks beyond `high` back to the global queue (warp-collective).
__device__ __forceinline__ int pool_spill(const KParams& P, uint32_t* fstack, int ftop, int high) {
    if (ftop - kChunk < high) return ftop;
    const int k = (ftop - high) / kChunk;
    __syncwarp();
    if (cq_push_many(P, fstack + ftop - k * kChunk, k)) ftop -= k * kChunk;
    return ftop;
}

// ---------------------------------------------------------------------------
// Per-warp shared-memory layout (thread mode).
struct WarpSh {
    int* ctrl;          // [0] ftop  [1] nfreed  [2] nstaged  [3] error
    int* cls_count;     // [kMaxQueues]
    uint32_t* tail;     // [kMaxQueues] owner tails (Sec. 5.1.3: tail kept in shared memory)
    int* push_off;      // [kMaxQueues]
    int* hint;          // [kMaxQueues] owner's upper bound of count (only the owner increases count)
    uint32_t* head_lb;  // [kMaxQueues] owner's lower bound of head (heads only grow)
    uint32_t* retained; // [32]
    uint32_t* freed;    // [32]
    uint32_t* fstack;   // [fcap]
    uint32_t* staged_id;// [scap]
    uint8_t* staged_q;  // [scap]
    char* prog;         // the program set's per-warp area (thread_prog_smem bytes, 16-byte aligned)
    int fcap, scap;
};

__device__ __forceinline__ WarpSh carve_warp(char* base, int maxspawn) {
    WarpSh w;
    w.fcap = thread_fcap(maxspawn);
    w.scap = thread_scap(maxspawn);
    int* ints = reinterpret_cast<int*>(base);
    w.ctrl = ints;
    w.cls_count = ints + 8;
    w.tail = reinterpret_cast<uint32_t*>(ints + 16);
    w.push_off = ints + 24;
    w.hint = ints + 32;
    w.head_lb = reinterpret_cast<uint32_t*>(ints + 40);
    w.retained = reinterpret_cast<uint32_t*>(base + 256);
    w.freed = reinterpret_cast<uint32_t*>(base + 384);
    w.fstack = reinterpret_cast<uint32_t*>(base + 512);
    w.staged_id = w.fstack + w.fcap;
    w.staged_q = reinterpret_cast<uint8_t*>(w.staged_id + w.scap);
    w.prog = base + thread_warp_smem(maxspawn);
    return w;
}

// ---------------------------------------------------------------------------
// Thread-mode task context: what a task program sees while one lane runs one
// step of one task (Sec. 4.2: one task per CUDA thread).
struct TaskCtx {
    const KParams& P;
    const WarpSh& ws;
    uint32_t self;
    FrameHdr h;
    char* frame;
    int worker;
    int nspawned;
    bool freed_self;
    bool staged_self = false;
    uint32_t iter = 0;

    uint4 pre[2];   // record bytes 16..47 (payload start), loaded together with the header

    // The header and the first 32 payload bytes are read in one burst of three
    // independent 16-byte loads, so the step waits for one L2 round trip, not two.
    __device__ TaskCtx(const KParams& p, const WarpSh& w, uint32_t id, int wk)
        : P(p), ws(w), self(id), frame(frame_ptr(p, id)), worker(wk), nspawned(0), freed_self(false) {
        const uint4* f4 = reinterpret_cast<const uint4*>(frame);
        const uint4 r0 = __ldcg(f4);
        pre[0] = __ldcg(f4 + 1);
        pre[1] = __ldcg(f4 + 2);
        memcpy(&h, &r0, sizeof(h));
    }
    __device__ int type() const { return (int)(h.w0 & 0xFF); }
    __device__ int pc() const { return (int)((h.w0 >> 8) & 0xFF); }
    template <class T> __device__ T* payload() const { return reinterpret_cast<T*>(frame + kHdrBytes); }
    // The payload as of the start of the step (children's results included).
    template <class T> __device__ T load() const {
        static_assert(sizeof(T) % 8 == 0, "payloads are 8-byte multiples");
        constexpr int kPre = (int)sizeof(pre);
        unsigned char buf[sizeof(T)];
        memcpy(buf, pre, sizeof(T) < (size_t)kPre ? sizeof(T) : (size_t)kPre);
        if constexpr (sizeof(T) > (size_t)kPre) {
#pragma unroll
            for (int o = kPre; o < (int)sizeof(T); o += 8) {
                const unsigned long long v = ld_cg64(frame + kHdrBytes + o);
                memcpy(buf + o, &v, 8);
            }
        }
        T out;
        memcpy(&out, buf, sizeof(T));
        return out;
    }
    // 8-byte word K of the record (a result slot) as of the start of the step.
    template <int K> __device__ unsigned long long word() const {
        static_assert(K >= 2, "words 0 and 1 are the header");
        if constexpr (K < 6) {
            unsigned long long v;
            memcpy(&v, reinterpret_cast<const unsigned char*>(pre) + 8 * (K - 2), 8);
            return v;
        } else {
            return ld_cg64(frame + 8 * K);
        }
    }

    __device__ void fail(int code, unsigned long long detail) { raise_error(P, code, type(), worker, detail); }

    __device__ uint32_t alloc() {
        int t = atomicSub(&ws.ctrl[0], 1) - 1;
        if (t < 0) return kNoTask;
        return ws.fstack[t];
    }
    __device__ void stage(uint32_t id, int q) {
        if (P.fstate != nullptr && dbg_stage_check(P, id, self, h.parent, worker)) staged_self = true;
        dbg_log(P, id, 2, worker, iter, id == self ? 1u : (id == h.parent ? 2u : 0u));
        q = (P.n_queues > 1) ? (int)((unsigned)q % P.n_queues) : 0;
        int p = atomicAdd(&ws.ctrl[2], 1);
        if (p >= ws.scap) { fail(GTAP_ERR_DEQUE_OVERFLOW, (unsigned long long)ws.scap); return; }
        ws.staged_id[p] = id;
        ws.staged_q[p] = (uint8_t)q;
        if (P.n_queues > 1) atomicAdd(&ws.cls_count[q], 1);
    }

    // Fork: create a child record (arguments copied now, Sec. 4.1) and stage it.
    // slot8 = byte offset / 8 of the parent-record word that receives the result.
    template <class A>
    __device__ void spawn(int type, uint32_t slot8, int q, const A& a, uint32_t flags = 0, uint32_t aux = 0) {
        static_assert(sizeof(A) % 4 == 0, "args must be 4-byte multiples");
        uint32_t id = alloc();
        if (id == kNoTask) { fail(GTAP_ERR_POOL_EXHAUSTED, P.n_frames); return; }
        if (kHdrBytes + sizeof(A) > P.frame_bytes) { fail(GTAP_ERR_INVALID_ARG, sizeof(A)); return; }
        dbg_transition(P, id, 0u, 1u, DBG_DOUBLE_ALLOC, type, worker);
        dbg_log(P, id, 1, worker, iter, self & 0xFFFF);
        char* f = frame_ptr(P, id);
        FrameHdr ch;
        ch.w0 = (uint32_t)type | (flags << 16);
        ch.pending = 0;
        ch.parent = self;
        ch.w3 = (slot8 & 0xFFFFu) | (aux << 16);
        st_obj(f, ch);
        st_obj(f + kHdrBytes, a);
        stage(id, q);
        ++nspawned;
    }

    // Join (taskwait): wait for the children spawned in this step, then resume
    // at pc_next on queue q_cont (the continuation is routed like a new task,
    // Sec. 5.1.2).  The waiting-child count is stored before any child is
    // published (children are published only after the step), so no
    // child can decrement it early.
    __device__ void join(int pc_next, int q_cont) {
        uint32_t w0 = (h.w0 & ~0xFF00u) | ((uint32_t)pc_next << 8);
        uint32_t pend = (uint32_t)nspawned | ((uint32_t)((P.n_queues > 1) ? ((unsigned)q_cont % P.n_queues) : 0) << 24);
        uint2 v = make_uint2(w0, pend);
        __stcg(reinterpret_cast<uint2*>(frame), v);
        dbg_log(P, self, 11, worker, iter, (unsigned)nspawned | ((unsigned)pc_next << 8));
        h.w0 = w0;
        if (nspawned == 0) stage(self, q_cont);
    }

    // Complete: deliver the result to the parent's slot (store, or atomic add
    // for accumulating programs), then decrement its waiting-child counter
    // with acq_rel ordering; the child that brings it to zero re-enqueues the
    // parent (Sec. 5.1.2).  The record is then freed.
    __device__ void ret(unsigned long long v) {
        const uint32_t parent = h.parent;
        const uint32_t slot = h.w3 & 0xFFFFu;
        const uint32_t flags = (h.w0 >> 16) & 0xFFu;
        if (parent & kRootBit) {
            RootEntry* r = &P.roots[parent & ~kRootBit];
            if (P.serving) {
                // served request: publish the result in the host-mapped outbox
                const unsigned long long pos = atomicAdd(&P.ctl->out_tail.v, 1ull);
                volatile OutboxEntry* o = P.outbox + (pos % P.outbox_cap);
                o->req = ld_cg64(&r->req);
                o->result[0] = v;
                o->result[1] = 0;
                o->status = 0;
                __threadfence_system();
                o->seq = pos + 1;
                __threadfence_system();
                atomicAdd(&P.ctl->inflight.v, ~0ull);
                // every task of the request has completed: its root slot may be reused
                st_release_u32(&r->done, kRootSlotFree);
            } else {
                if (flags & kFlagAccumulate) atomicAdd(&r->result[slot & 1], v);
                else st_cg64(&r->result[slot & 1], v);
                __threadfence();
                atomicExch(&r->done, 1u);
                atomicAdd(&P.ctl->roots_remaining.v, ~0ull);
            }
        } else {
            char* pf = frame_ptr(P, parent);
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(pf + slot * 8);
            if (flags & kFlagAccumulate) { if (v) atomicAdd(dst, v); }
            else st_cg64(dst, v);
            uint32_t old = atom_add_acqrel_u32(pf + 4, 0xFFFFFFFFu);
            dbg_log(P, parent, 10, worker, iter, (old & 0xFF) | ((self & 0xFF) << 8));
            if ((old & 0xFFFFFFu) == 1u) stage(parent, (int)(old >> 24));
        }
        dbg_log(P, self, 5, worker, iter, 0);
        dbg_transition(P, self, 2u, 0u, DBG_DOUBLE_FREE, type(), worker);
        int p = atomicAdd(&ws.ctrl[1], 1);
        ws.freed[p] = self;
        freed_self = true;
    }
};

// ---------------------------------------------------------------------------
// Serving: warp 0 of the grid is the inbox poller.  It admits a request when
// enough task records are free and the outbox has room, writes the request's
// root record (frames from the pool, environment into the root table slot),
// and pushes it on its own deque, from which the other warps steal it.
// Requests that arrive while others run are admitted as records and root
// slots free up, so their work overlaps on the device (continuous batching).
static __device__ __noinline__ void serve_poller(const KParams& P, const WarpSh& ws, int* ftop_io) {
    const int lane = threadIdx.x & 31;
    const int Q = (int)P.n_queues;
    const uint32_t cap_mask = P.ring_mask;
    QState* myq = P.qs;                       // warp 0's queues
    uint32_t* myring = P.rings;
    int ftop = *ftop_io;
    unsigned long long next = 0;              // next inbox sequence to take
    int backoff = 64;
    // a root slot is free when its `done` word holds kRootSlotFree (completions
    // release it); the poller is the only taker, so a slot it found free stays
    // free until it admits a request into it
    int rslot = -1;
    uint32_t cursor = 0;
    for (uint32_t iter = 0;; ++iter) {
        ftop = pool_refill(P, ws.fstack, ftop, 32);
        if (rslot < 0) {
            const uint32_t cand = (cursor + (uint32_t)lane) % P.n_roots;
            const bool fr = ld_acquire_u32(&P.roots[cand].done) == kRootSlotFree;
            const unsigned m = __ballot_sync(0xffffffffu, fr);
            if (m) {
                rslot = (int)((cursor + (uint32_t)(__ffs((int)m) - 1)) % P.n_roots);
                cursor = ((uint32_t)rslot + 1u) % P.n_roots;
            } else {
                cursor = (cursor + 32u) % P.n_roots;
            }
        }
        int stop = 0, took = 0;
        if (lane == 0) {
            volatile HostFlags* hf = P.hflags;
            if (ld_cg64(&P.ctl->abort_flag.v) != 0 || hf->abort != 0) {
                stop = 1;
            } else {
                volatile InboxSlot* slot = P.inbox + (next % P.inbox_cap);
                const unsigned long long sq = slot->seq;
                if (sq == next + 1) {
                    __threadfence_system();
                    const unsigned long long bump = ld_cg64(&P.ctl->bump.v);
                    const unsigned long long used = bump < P.n_frames ? bump : P.n_frames;
                    const unsigned long long free_records = (P.n_frames - used) + 32ull * ld_cg64(&P.ctl->cq_avail.v);
                    const unsigned long long inflight = ld_cg64(&P.ctl->inflight.v);
                    const unsigned long long unread = ld_cg64(&P.ctl->out_tail.v) - hf->out_consumed;
                    const uint32_t q = slot->queue % (uint32_t)Q;
                    const bool room = ws.tail[q] - ws.head_lb[q] + 1u <= cap_mask + 1 ||
                                      ws.tail[q] - (ws.head_lb[q] = __ldcg(&myq[q].head)) + 1u <= cap_mask + 1;
                    if (free_records >= P.admit_reserve && ftop > 0 && inflight < P.n_roots && rslot >= 0 &&
                        inflight + unread < P.outbox_cap && room) {
                        const uint32_t r = (uint32_t)rslot;
                        const uint32_t id = ws.fstack[--ftop];
                        const uint32_t type = slot->type;
                        // root environment (read by programs with per-root buffers)
                        RootDesc* d = const_cast<RootDesc*>(P.root_desc) + r;
                        for (int i = 0; i < kRootArgBytes / 4; ++i)
                            st_cg32(d->env + 4 * i, ((volatile uint32_t*)slot->env)[i]);
                        char* f = frame_ptr(P, id);
                        FrameHdr h;
                        h.w0 = type & 0xFFu;
                        h.pending = 0;
                        h.parent = kRootBit | r;
                        h.w3 = 0;
                        st_obj(f, h);
                        for (int i = 0; i < kRootPayloadBytes / 4; ++i) {
                            uint32_t w = ((volatile uint32_t*)slot->payload)[i];
                            if (i == 0 && type == T_KCLIQUE_ROOT) w = r;   // programs with a root environment name its slot
                            st_cg32(f + kHdrBytes + 4 * i, w);
                        }
                        RootEntry e;
                        e.result[0] = 0; e.result[1] = 0; e.done = 0; e.type = type; e.req = next;
                        st_obj(&P.roots[r], e);
                        // push on the poller's own deque (one fence, one count increment)
                        const uint32_t t = ws.tail[q];
                        __stcg(&myring[(size_t)q * (cap_mask + 1) + (t & cap_mask)], id);
                        __threadfence();
                        atomicAdd(&P.ctl->inflight.v, 1ull);
                        atomicAdd(&P.ctl->admitted.v, 1ull);
                        ws.tail[q] = t + 1u;
                        atomicAdd(&myq[q].count, 1);
                        hf->inbox_consumed = next + 1;
                        ++next;
                        took = 1;
                    }
                } else {
                    const unsigned long long sd = hf->shutdown;
                    if (sd != 0 && next == sd - 1) stop = 1;   // the host closed the inbox and all is taken
                }
            }
        }
        stop = __shfl_sync(0xffffffffu, stop, 0);
        took = __shfl_sync(0xffffffffu, took, 0);
        ftop = __shfl_sync(0xffffffffu, ftop, 0);
        if (stop) break;
        if (took) {
            rslot = -1;
            backoff = 64;
        } else {
            __nanosleep(backoff);
            backoff = min(backoff * 2, 1024);
        }
    }
    *ftop_io = ftop;
}

// ---------------------------------------------------------------------------
// Thread-mode scheduler loop (Algorithm 1), one instance per warp.
// Dispatch is a functor: Dispatch::run(TaskCtx&) executes one step.
// The longest sleep of an idle warp between steal rounds is a configuration
// field (default 512 ns): longer sleeps relieve L2 of idle probing (the hashed
// tree gained 8 % at 4 us) but slow the spread of work at start-up (fib and
// N-Queens lost 15-25 % at 4 us), so the autotuner picks it per program.

template <class Dispatch, int SCHED = SCHED_BATCHED>
__device__ void thread_mode_loop(const KParams& P, char* smem_warp) {
    const int lane = threadIdx.x & 31;
    const int wid = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    const int Q = (int)P.n_queues;
    const uint32_t cap_mask = P.ring_mask;
    WarpSh ws = carve_warp(smem_warp, (int)P.maxspawn);

    QState* myq = P.qs + (size_t)wid * Q;
    uint32_t* myring = P.rings + (size_t)wid * Q * (cap_mask + 1);
    if (lane < 8) {
        ws.cls_count[lane] = 0;
        ws.push_off[lane] = 0;
        const uint32_t t0 = (lane < Q) ? __ldcg(&myq[lane].tail0) : 0u;
        ws.tail[lane] = t0;
        ws.hint[lane] = (int)t0;   // the reset kernel leaves count == tail0 and head == 0
        ws.head_lb[lane] = 0;
    }
    if (lane == 0) { ws.ctrl[0] = 0; ws.ctrl[1] = 0; ws.ctrl[2] = 0; ws.ctrl[3] = 0; }
    {
        // the program set's warp area starts zeroed
        const int pwords = ((int)P.warp_smem - thread_warp_smem((int)P.maxspawn)) / 4;
        for (int i = lane; i < pwords; i += 32) reinterpret_cast<int*>(ws.prog)[i] = 0;
    }
    __syncwarp();

    if (P.serving && wid == 0) {
        int ft = 0;
        serve_poller(P, ws, &ft);
        if (lane == 0) { WorkerStats s{}; P.stats[wid] = s; }
        return;
    }
    unsigned long long st_tasks = 0, st_steps = 0, st_pops = 0, st_popped = 0, st_sa = 0, st_steals = 0,
                       st_stolen = 0, st_idle = 0, st_pushes = 0, st_pushed = 0, st_spawned = 0;
    // per-lane xorshift state for victim probing
    uint64_t rng = P.seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(wid + 1)) ^ (0xD1B54A32D192ED03ull * (uint64_t)(lane + 1));
    const uint64_t t_start = global_ns();
    const uint64_t deadline = t_start + P.timeout_ns;
    uint32_t tid = kNoTask;  // this lane's task (valid for lane < cnt)
    int src = 0;             // debug: where tid came from (0 retained, 1 popped, 2 stolen)
    int cnt = 0;             // warp-uniform: lanes holding a task
    int cls = 0;             // warp-uniform: DAQ queue of the current batch
    int backoff = 32;
    int ftop = 0;
    const int fhigh = 32 * (int)P.maxspawn + 2 * kChunk;
    constexpr int kProbes = 8;   // victims probed in parallel per steal attempt (one lane each)
    // Fill steals (the warp holds tasks but fewer than 32) back off after failures:
    // after k failed attempts in a row the next 2^k - 1 steps skip them (k <= 6).
    // A warp with no task at all always tries.  Warp-uniform.
    int fill_fail = 0, fill_wait = 0;
    // per-phase clock accounting (tracing counters): pop, steal, execute, retain/push, idle
    unsigned long long cy_pop = 0, cy_steal = 0, cy_exec = 0, cy_push = 0, cy_idle = 0;
    long long tc0 = clock64();

    for (uint32_t iter = 0;; ++iter) {
        if ((iter & 63u) == 0u) {
            int ab = 0;
            if (lane == 0) ab = abort_requested(P, (iter & 1023u) == 0u) ? 1 : 0;
            if (__shfl_sync(0xffffffffu, ab, 0)) break;
        }
        if constexpr (SCHED == SCHED_GLOBAL) {
            // ---- Central queue (Sec. 6.5 comparison): the warp claims up to 32 - cnt tasks
            // from the one queue every warp shares (reserve from the published count, then
            // take dequeue tickets; each lane waits for its slot's publication).
            if (cnt < 32) {
                const int want = 32 - cnt;
                int got = 0;
                unsigned long long d0 = 0;
                if (lane == 0 && (long long)ld_cg64(&P.ctl->gq_avail.v) > 0) {
                    const long long av = (long long)atomicAdd(&P.ctl->gq_avail.v, (unsigned long long)(-(long long)want));
                    got = (int)max(0ll, min((long long)want, av));
                    if (got < want) atomicAdd(&P.ctl->gq_avail.v, (unsigned long long)(want - got));
                    if (got > 0) d0 = atomicAdd(&P.ctl->gq_deq.v, (unsigned long long)got);
                }
                got = __shfl_sync(0xffffffffu, got, 0);
                d0 = __shfl_sync(0xffffffffu, d0, 0);
                if (got > 0) {
                    int bad = 0;
                    if (lane >= cnt && lane < cnt + got) {
                        const unsigned long long tk = d0 + (unsigned long long)(lane - cnt);
                        unsigned long long* slot = &P.gq[tk & P.gq_mask];
                        bad = 1;
                        for (int it = 0; it < (1 << 20); ++it) {
                            const unsigned long long w = ld_acquire_u64(slot);
                            if ((uint32_t)(w >> 32) == (uint32_t)(tk + 1)) {
                                tid = (uint32_t)w;
                                st_release_u64(slot, (unsigned long long)(uint32_t)(tk + P.gq_mask + 1) << 32);
                                bad = 0;
                                break;
                            }
                            __nanosleep(32);
                        }
                        if (bad) raise_error(P, GTAP_ERR_TASK_FAILED, -1, wid, tk);
                        src = 1;
                    }
                    if (__any_sync(0xffffffffu, bad)) break;
                    cnt += got;
                    cls = 0;
                    ++st_pops;
                    st_popped += got;
                }
            }
        } else if constexpr (SCHED == SCHED_SINGLE) {
            // ---- Non-batched pop (Sec. 6.5 comparison): single-task claims, one CAS each,
            // issued one after another by lane 0 until the batch is full or the queue is empty.
            const int q = 0;
            if (cnt < 32 && ws.hint[q] > 0) {
                int claim = 0;
                if (lane == 0) {
                    int old = ws.hint[q];
                    for (int k = 0; k < 32 - cnt && old > 0; ++k) {
                        bool ok = false;
                        for (int it = 0; it < 64 && old > 0; ++it) {
                            const int got = atom_cas_acq_i32(&myq[q].count, old, old - 1);
                            if (got == old) { ok = true; old -= 1; break; }
                            old = got;
                        }
                        if (!ok) break;
                        const uint32_t t = ws.tail[q] - 1u;
                        ws.tail[q] = t;
                        ws.retained[cnt + claim] = __ldcg(&myring[t & cap_mask]);
                        ++claim;
                    }
                    ws.hint[q] = max(old, 0);
                }
                claim = __shfl_sync(0xffffffffu, claim, 0);
                __syncwarp();
                if (claim > 0) {
                    if (lane >= cnt && lane < cnt + claim) { tid = ws.retained[lane]; src = 1; }
                    cnt += claim;
                    cls = 0;
                    st_pops += claim;
                    st_popped += claim;
                }
                __syncwarp();
            }
        } else {
            // ---- PopBatch (Algorithm 2) from the own queue: the retained class, else the fullest (DAQ).
            // The owner keeps an upper bound of each count (thieves only lower it), so an empty
            // queue costs no memory access and the CAS starts from a good guess.
            if (cnt < 32) {
                int q = cls;
                if (cnt == 0 && Q > 1) {
                    int best = (lane < Q) ? ws.hint[lane] : -1, bq = lane;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        int oc = __shfl_down_sync(0xffffffffu, best, o);
                        int oq = __shfl_down_sync(0xffffffffu, bq, o);
                        if (oc > best || (oc == best && oq < bq)) { best = oc; bq = oq; }
                    }
                    q = __shfl_sync(0xffffffffu, bq, 0);
                }
                if (ws.hint[q] > 0) {
                    int claim = 0;
                    if (lane == 0) {
                        int old = ws.hint[q];
                        for (int it = 0; it < 64 && old > 0; ++it) {
                            const int want = min(32 - cnt, old);
                            const int got = atom_cas_acq_i32(&myq[q].count, old, old - want);
                            if (got == old) { claim = want; old -= want; break; }
                            old = got;
                        }
                        ws.hint[q] = max(old, 0);
                    }
                    claim = __shfl_sync(0xffffffffu, claim, 0);
                    if (claim > 0) {
                        uint32_t t = ws.tail[q] - (uint32_t)claim;
                        if (lane >= cnt && lane < cnt + claim) {
                            uint32_t* slot = &myring[(size_t)q * (cap_mask + 1) + ((t + (uint32_t)(lane - cnt)) & cap_mask)];
                            tid = __ldcg(slot);
                            src = 1;
                            dbg_log(P, tid, 7, wid, iter, (t + (uint32_t)(lane - cnt)) & 0xFFFF);
                            if (P.fstate != nullptr) dbg_take_slot(P, slot, tid, 100 + 1, wid);
                        }
                        __syncwarp();
                        if (lane == 0) ws.tail[q] = t;
                        __syncwarp();
                        cnt += claim;
                        cls = q;
                        ++st_pops;
                        st_popped += claim;
                    } else {
                        __syncwarp();
                    }
                }
            }
        }
        { const long long t = clock64(); cy_pop += (unsigned long long)(t - tc0); tc0 = t; }
        // ---- StealBatch.  SelectVictimQueue probes kProbes random victims at once (one
        // lane each) and picks the fullest, so an idle warp finds work in one round trip.
        bool want_steal = (P.steal_policy & GTAP_STEAL_EMPTY) ? (cnt == 0) : (cnt < 32);
        if constexpr (SCHED == SCHED_GLOBAL) want_steal = false;   // no per-warp deques to steal from
        const bool fill = cnt > 0;
        if (want_steal && fill && fill_wait > 0) {
            --fill_wait;
            want_steal = false;
        }
        if (want_steal && P.n_workers > 1) {
            const int cnt_before = cnt;
            ++st_sa;
            int c = -1, victim = 0, vqi = cls;
            if (lane < kProbes) {
                rng ^= rng >> 12; rng ^= rng << 25; rng ^= rng >> 27;
                const uint64_t r = rng * 2685821657736338717ull;
                victim = (int)(((r >> 32) * (unsigned long long)(P.n_workers - 1)) >> 32);
                if (victim >= wid) ++victim;
                if (cnt == 0 && Q > 1) {
                    // a warp with no batch yet may take any class: read all of the victim's queues
                    int cc[kMaxQueues];
#pragma unroll
                    for (int k = 0; k < kMaxQueues; ++k) cc[k] = (k < Q) ? ld_cg_i32(&P.qs[(size_t)victim * Q + k].count) : -1;
#pragma unroll
                    for (int k = 0; k < kMaxQueues; ++k) if (cc[k] > c) { c = cc[k]; vqi = k; }
                } else {
                    c = ld_cg_i32(&P.qs[(size_t)victim * Q + vqi].count);
                }
            }
            int best = c, bl = lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                int oc = __shfl_down_sync(0xffffffffu, best, o);
                int ol = __shfl_down_sync(0xffffffffu, bl, o);
                if (oc > best) { best = oc; bl = ol; }
            }
            bl = __shfl_sync(0xffffffffu, bl, 0);
            best = __shfl_sync(0xffffffffu, best, 0);
            victim = __shfl_sync(0xffffffffu, victim, bl);
            const int q = __shfl_sync(0xffffffffu, vqi, bl);
            if (best > 0) {
                if constexpr (SCHED == SCHED_SINGLE) {
                    // non-batched steal (Sec. 6.5 comparison): lane 0 repeats single-task steals
                    // from the chosen victim, each one lock, one CAS, one head read and update
                    QState* vq = P.qs + (size_t)victim * Q + q;
                    const uint32_t* vring = P.rings + ((size_t)victim * Q + q) * (cap_mask + 1);
                    int claim = 0;
                    if (lane == 0) {
                        int old = best;
                        for (int k = 0; k < 32 - cnt && old > 0; ++k) {
                            if (atom_cas_acq_i32(&vq->lock, 0, 1) != 0) break;   // try-lock
                            bool ok = false;
                            for (int it = 0; it < 64 && old > 0; ++it) {
                                const int got = atom_cas_acq_i32(&vq->count, old, old - 1);
                                if (got == old) { ok = true; old -= 1; break; }
                                old = got;
                            }
                            if (ok) {
                                const uint32_t hd = __ldcg(&vq->head);
                                const uint32_t id = __ldcg(&vring[hd & cap_mask]);
                                uint32_t zero;
                                asm volatile("and.b32 %0, %1, 0;" : "=r"(zero) : "r"(id));  // the head store waits for the load
                                __threadfence();
                                __stcg(&vq->head, hd + 1u + zero);
                                ws.retained[cnt + claim] = id;
                                ++claim;
                            }
                            st_release_i32(&vq->lock, 0);
                            if (!ok) break;
                        }
                    }
                    claim = __shfl_sync(0xffffffffu, claim, 0);
                    __syncwarp();
                    if (claim > 0) {
                        if (lane >= cnt && lane < cnt + claim) { tid = ws.retained[lane]; src = 2; }
                        cnt += claim;
                        cls = q;
                        st_steals += claim;
                        st_stolen += claim;
                    }
                    __syncwarp();
                } else {
                    QState* vq = P.qs + (size_t)victim * Q + q;
                    int claim = 0;
                    uint32_t h = 0;
                    if (lane == 0) {
                        if (atom_cas_acq_i32(&vq->lock, 0, 1) == 0) {  // try-lock: never wait on a thief
                            int old = best;
                            for (int it = 0; it < 64 && old > 0; ++it) {
                                int want = min(32 - cnt, old);
                                if (P.steal_policy & GTAP_STEAL_HALF) want = min(want, (old + 1) >> 1);
                                const int got = atom_cas_acq_i32(&vq->count, old, old - want);
                                if (got == old) { claim = want; break; }
                                old = got;
                            }
                            if (claim > 0) h = __ldcg(&vq->head);
                            else st_release_i32(&vq->lock, 0);
                        }
                    }
                    claim = __shfl_sync(0xffffffffu, claim, 0);
                    if (claim > 0) {
                        h = __shfl_sync(0xffffffffu, h, 0);
                        const uint32_t* vring = P.rings + ((size_t)victim * Q + q) * (cap_mask + 1);
                        if (lane >= cnt && lane < cnt + claim) {
                            uint32_t* slot = const_cast<uint32_t*>(&vring[(h + (uint32_t)(lane - cnt)) & cap_mask]);
                            tid = __ldcg(slot);
                            src = 2;
                            dbg_log(P, tid, 8, wid, iter, (unsigned)victim & 0xFFFF);
                            if (P.fstate != nullptr) dbg_take_slot(P, slot, tid, 100 + 2, wid);
                        }
                        // every claimed ID is in a register before the head moves (wrap-around safety, Sec. 5.1.3)
                        const uint32_t used = __reduce_or_sync(0xffffffffu, (lane >= cnt && lane < cnt + claim) ? tid : 0u);
                        uint32_t zero;
                        asm volatile("and.b32 %0, %1, 0;" : "=r"(zero) : "r"(used));  // the head store waits for the loads
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) {
                            __stcg(&vq->head, h + (uint32_t)claim + zero);
                            st_release_i32(&vq->lock, 0);
                        }
                        cnt += claim;
                        cls = q;
                        ++st_steals;
                        st_stolen += claim;
                    }
                }
            }
            if (fill) {
                if (cnt > cnt_before) {
                    fill_fail = 0;
                } else {
                    fill_fail = min(fill_fail + 1, 6);
                    fill_wait = (1 << fill_fail) - 1;
                }
            }
        }
        { const long long t = clock64(); cy_steal += (unsigned long long)(t - tc0); tc0 = t; }
        // ---- Nothing to run: termination test (all roots complete), deadline, backoff.
        if (cnt == 0) {
            ++st_idle;
            int stop = 0;
            if (lane == 0 && (st_idle & 15ull) == 1ull) {
                if (P.serving) {
                    // served session: done once the host has closed the inbox, every submitted
                    // request has been admitted and none is in flight
                    const unsigned long long sd = *(volatile unsigned long long*)&P.hflags->shutdown;
                    if (sd != 0 && ld_cg64(&P.ctl->admitted.v) == sd - 1 && ld_cg64(&P.ctl->inflight.v) == 0) stop = 1;
                } else if (ld_cg64(&P.ctl->roots_remaining.v) == 0ull) stop = 1;
                else if (abort_requested(P, (st_idle & 255ull) == 1ull)) stop = 1;
                else if (!P.serving && global_ns() > deadline) { raise_error(P, GTAP_ERR_TIMEOUT, -1, wid, P.timeout_ns); stop = 1; }
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) break;
            __nanosleep(backoff);
            backoff = min(backoff * 2, P.idle_backoff_ns);
            { const long long t = clock64(); cy_idle += (unsigned long long)(t - tc0); tc0 = t; }
            continue;
        }
        backoff = 32;

        // ---- Ensure the free stack can serve every spawn of this step.
        ftop = pool_refill(P, ws.fstack, ftop, cnt * (int)P.maxspawn);
        if (lane == 0) { ws.ctrl[0] = ftop; ws.ctrl[1] = 0; ws.ctrl[2] = 0; }
        if (lane < 8) ws.cls_count[lane] = 0;
        __syncwarp();

        // ---- Execute: lanes [0, cnt) run one step of their task.
        int spawned = 0;
        if (lane < cnt) {
            if (P.fstate != nullptr) dbg_exec_check(P, tid, src, wid);
            TaskCtx c(P, ws, tid, wid);
            c.iter = iter;
            dbg_log(P, tid, 3, wid, iter, (unsigned)c.pc() | ((unsigned)src << 8));
            Dispatch::run(c);
            spawned = c.nspawned;
            if (!c.freed_self) dbg_log(P, tid, 4, wid, iter, 0);
            if (!c.freed_self && !c.staged_self) dbg_transition(P, tid, 2u, 1u, DBG_EXEC_NOT_ALLOCATED, c.type(), wid);
        }
        __syncwarp();
        st_spawned += (unsigned)__reduce_add_sync(0xffffffffu, (unsigned)spawned);
        st_tasks += cnt;
        ++st_steps;
        { const long long t = clock64(); cy_exec += (unsigned long long)(t - tc0); tc0 = t; }

        // ---- Return freed records to the local stack; spill the surplus.
        {
            int top = max(ws.ctrl[0], 0);
            int nf = ws.ctrl[1];
            __syncwarp();
            // the cache never exceeds its capacity (a spill that could not run leaves the surplus out)
            nf = min(nf, ws.fcap - top);
            if (lane < nf) ws.fstack[top + lane] = ws.freed[lane];
            __syncwarp();
            ftop = pool_spill(P, ws.fstack, top + nf, fhigh);
        }

        // ---- Retain up to 32 staged tasks of one queue class; push the rest (PushBatch).
        const int nst = ws.ctrl[2];
        cnt = 0;
        if (nst > 0) {
            int qstar = 0, nq_star = nst;
            if (Q > 1) {
                // DAQ: the next batch is the class with the most runnable work this warp holds
                // (staged now plus its own queue), so batches stay both homogeneous and full
                int c = (lane < Q) ? ws.cls_count[lane] + ws.hint[lane] : -1;
                if (lane < Q && ws.cls_count[lane] == 0) c = -1;   // only classes with staged tasks can be retained
                int best = c, bq = lane;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    int oc = __shfl_down_sync(0xffffffffu, best, o);
                    int oq = __shfl_down_sync(0xffffffffu, bq, o);
                    if (oc > best || (oc == best && oq < bq)) { best = oc; bq = oq; }
                }
                qstar = __shfl_sync(0xffffffffu, bq, 0);
                nq_star = ws.cls_count[qstar];
            }
            const int nkeep = min(32, nq_star);
            // capacity check per destination queue: uses head/tail, not count (Sec. 5.1.3)
            int overflow = 0;
            if (lane < Q) {
                int npush = ((Q > 1) ? ws.cls_count[lane] : nst) - (lane == qstar ? nkeep : 0);
                // (the central queue has a slot for every record, so it cannot overflow)
                if (SCHED != SCHED_GLOBAL && npush > 0 && ws.tail[lane] - ws.head_lb[lane] + (uint32_t)npush > cap_mask + 1) {
                    const uint32_t hd = __ldcg(&myq[lane].head);   // refresh the lower bound only when needed
                    ws.head_lb[lane] = hd;
                    if (ws.tail[lane] - hd + (uint32_t)npush > cap_mask + 1) overflow = 1;
                }
                ws.push_off[lane] = 0;
            }
            if (__any_sync(0xffffffffu, overflow)) {
                if (lane == 0) raise_error(P, GTAP_ERR_DEQUE_OVERFLOW, -1, wid, cap_mask + 1);
                break;
            }
            __syncwarp();
            unsigned long long gt0 = 0;   // central queue: first enqueue ticket of this batch
            if constexpr (SCHED == SCHED_GLOBAL) {
                // the records must be visible before any slot publishes them
                if (nkeep < nst) {
                    __threadfence();
                    if (lane == 0) gt0 = atomicAdd(&P.ctl->gq_enq.v, (unsigned long long)(nst - nkeep));
                    gt0 = __shfl_sync(0xffffffffu, gt0, 0);
                }
                __syncwarp();
            }
            int kept = 0;
            int gbad = 0;
            for (int base = 0; base < nst; base += 32) {
                const int i = base + lane;
                const bool valid = i < nst;
                uint32_t id = valid ? ws.staged_id[i] : kNoTask;
                int q = valid ? (int)ws.staged_q[i] : 0;
                const bool cand = valid && q == qstar;
                const uint32_t km = __ballot_sync(0xffffffffu, cand);
                const int rk = __popc(km & lanemask_lt());
                const bool keep = cand && (kept + rk) < nkeep;
                if (keep) { ws.retained[kept + rk] = id; dbg_log(P, id, 9, wid, iter, (unsigned)(kept + rk)); }
                kept = min(nkeep, kept + __popc(km));
                const bool push = valid && !keep;
                const uint32_t key = push ? (uint32_t)q : (0x100u + (uint32_t)lane);
                const uint32_t grp = __match_any_sync(0xffffffffu, key);
                const int prk = __popc(grp & lanemask_lt());
                int off = 0;
                if (push) off = ws.push_off[q];
                __syncwarp();
                if (push) {
                    if constexpr (SCHED == SCHED_GLOBAL) {
                        // wait (bounded) for the slot's previous occupant to be taken, then publish
                        const unsigned long long tk = gt0 + (unsigned long long)(off + prk);
                        unsigned long long* slot = &P.gq[tk & P.gq_mask];
                        int ok = 0;
                        for (int it = 0; it < (1 << 20); ++it) {
                            if ((uint32_t)(ld_acquire_u64(slot) >> 32) == (uint32_t)tk) { ok = 1; break; }
                            __nanosleep(32);
                        }
                        if (ok) st_release_u64(slot, ((unsigned long long)(uint32_t)(tk + 1) << 32) | id);
                        else { gbad = 1; raise_error(P, GTAP_ERR_TASK_FAILED, -1, wid, tk); }
                    } else {
                        uint32_t pos = ws.tail[q] + (uint32_t)(off + prk);
                        __stcg(&myring[(size_t)q * (cap_mask + 1) + (pos & cap_mask)], id);
                        dbg_log(P, id, 6, wid, iter, pos & 0xFFFF);
                    }
                    if (prk == 0) ws.push_off[q] = off + __popc(grp);
                }
                __syncwarp();
            }
            // one fence, then one count increment per destination queue (PushBatch).  When every
            // staged task is retained nothing is published to other warps, so no fence is needed:
            // the warp's own lanes see the records through the warp barrier.
            if constexpr (SCHED == SCHED_GLOBAL) {
                if (__any_sync(0xffffffffu, gbad)) break;
                __syncwarp();
                if (lane == 0 && nkeep < nst) atomicAdd(&P.ctl->gq_avail.v, (unsigned long long)(nst - nkeep));
            } else {
                if (nkeep < nst) __threadfence();
                __syncwarp();
                if (lane < Q) {
                    int np = ws.push_off[lane];
                    if (np > 0) {
                        ws.tail[lane] += (uint32_t)np;
                        ws.hint[lane] += np;
                        atomicAdd(&myq[lane].count, np);
                    }
                }
            }
            if (lane == 0) {
                int tot = 0;
                for (int q = 0; q < Q; ++q) tot += ws.push_off[q];
                if (tot > 0) { ++st_pushes; st_pushed += tot; }
            }
            __syncwarp();
            if (lane < nkeep) { tid = ws.retained[lane]; src = 0; }
            cnt = nkeep;
            cls = qstar;
            __syncwarp();
        }
        { const long long t = clock64(); cy_push += (unsigned long long)(t - tc0); tc0 = t; }
    }

    // Give cached frames back so a later run or another worker could use them (best effort).
    if (lane == 0) {
        WorkerStats s;
        s.tasks = st_tasks; s.steps = st_steps; s.pops = st_pops; s.popped = st_popped;
        s.steal_attempts = st_sa; s.steals = st_steals; s.stolen = st_stolen; s.idle = st_idle;
        s.pushes = st_pushes; s.pushed = st_pushed; s.spawned = st_spawned;
        s.pad[0] = cy_pop; s.pad[1] = cy_steal; s.pad[2] = cy_exec; s.pad[3] = cy_push; s.pad[4] = cy_idle;
        P.stats[wid] = s;
    }
}


// ===========================================================================
// Block mode (Sec. 4.3, Sec. 5.1.3 "Block Mode"): one deque per block, a
// leader acquires at most one task by single-task pop or steal, and the whole
// block executes it.  The deque uses the same count-claim protocol as thread
// mode with claims of one entry.
struct BlockSh {
    int* ctrl;          // [0] ftop [2] nstaged [3] state (0 idle, 1 task, 2 exit) [4] join pc+1 [5] completed
    uint32_t* misc;     // [0] current task [1] retained task [2] own tail
    FrameHdr* hdr;      // header of the current task (the first 16 bytes of rec)
    uint4* rec;         // [8]: the current task's record bytes 0..127, read once by warp 0
    uint32_t* fstack;   // [fcap]
    uint32_t* staged_id;// [scap]
    char* prog;         // program shared area
    int fcap, scap;
};

__device__ __forceinline__ BlockSh carve_block(char* base, int step_max) {
    BlockSh b;
    b.fcap = block_fcap(step_max);
    b.scap = block_scap(step_max);
    b.ctrl = reinterpret_cast<int*>(base);
    b.misc = reinterpret_cast<uint32_t*>(base + 32);
    b.rec = reinterpret_cast<uint4*>(base + 64);
    b.hdr = reinterpret_cast<FrameHdr*>(base + 64);
    b.fstack = reinterpret_cast<uint32_t*>(base + 192);
    b.staged_id = b.fstack + b.fcap;
    b.prog = reinterpret_cast<char*>(b.staged_id + b.scap);
    return b;
}

// Block-mode task context: all threads of the block run the same step.
struct BTaskCtx {
    const KParams& P;
    const BlockSh& bs;
    uint32_t self;
    FrameHdr h;
    char* frame;
    int worker;

    __device__ BTaskCtx(const KParams& p, const BlockSh& b, int wk)
        : P(p), bs(b), self(b.misc[0]), h(*b.hdr), frame(frame_ptr(p, b.misc[0])), worker(wk) {}
    __device__ int type() const { return (int)(h.w0 & 0xFF); }
    __device__ int pc() const { return (int)((h.w0 >> 8) & 0xFF); }
    // The payload, from the shared-memory copy of the record taken at acquire.
    template <class T> __device__ T load() const {
        static_assert(kHdrBytes + sizeof(T) <= 128, "block-mode payloads fit the first 128 record bytes");
        T out;
        memcpy(&out, reinterpret_cast<const unsigned char*>(bs.rec) + kHdrBytes, sizeof(T));
        return out;
    }
    template <class T> __device__ T* prog_smem() const { return reinterpret_cast<T*>(bs.prog); }
    __device__ void fail(int code, unsigned long long detail) { raise_error(P, code, type(), worker, detail); }

    // Per-thread fork (Sec. 4.3: the spawn is performed by each thread that reaches it).
    template <class A>
    __device__ void spawn(int type, uint32_t slot8, const A& a) {
        int t = atomicSub(&bs.ctrl[0], 1) - 1;
        if (t < 0) { fail(GTAP_ERR_POOL_EXHAUSTED, P.n_frames); return; }
        uint32_t id = bs.fstack[t];
        dbg_transition(P, id, 0u, 1u, DBG_DOUBLE_ALLOC, type, worker);
        char* f = frame_ptr(P, id);
        FrameHdr ch;
        ch.w0 = (uint32_t)type;
        ch.pending = 0;
        ch.parent = self;
        ch.w3 = (slot8 & 0xFFFFu) | ((uint32_t)threadIdx.x << 16);  // aux = spawning thread
        st_obj(f, ch);
        st_obj(f + kHdrBytes, a);
        int p = atomicAdd(&bs.ctrl[2], 1);
        if (p >= bs.scap - 1) { fail(GTAP_ERR_DEQUE_OVERFLOW, (unsigned long long)bs.scap); return; }
        bs.staged_id[p] = id;
    }
    // Block-collective join (taskwait must be reached by all threads, Sec. 4.3).
    __device__ void join(int pc_next) {
        if (threadIdx.x == 0) bs.ctrl[4] = pc_next + 1;
    }
    // Block-collective completion with per-thread return values: thread i of
    // the parent observes this task's thread i, and only on the thread that
    // executed the spawn (Sec. 4.3, "Values across spawn and join").
    __device__ void ret(unsigned long long v) {
        const uint32_t parent = h.parent;
        const uint32_t slot = h.w3 & 0xFFFFu;
        const uint32_t spawner = h.w3 >> 16;
        if (parent & kRootBit) {
            if (threadIdx.x == 0) st_cg64(&P.roots[parent & ~kRootBit].result[0], v);
        } else if (threadIdx.x == spawner && slot != 0) {
            st_cg64(frame_ptr(P, parent) + (size_t)slot * 8 + (size_t)spawner * 8, v);
        }
        __threadfence();
        if (threadIdx.x == 0) bs.ctrl[5] = 1;
    }
    __device__ void ret_void() {
        if (threadIdx.x == 0) bs.ctrl[5] = 1;
    }
};

template <class Dispatch>
__device__ void block_mode_loop(const KParams& P, char* smem, int bsz) {
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    const int bid = (int)blockIdx.x;
    const uint32_t cap_mask = P.ring_mask;
    BlockSh bs = carve_block(smem, (int)P.maxspawn);
    QState* myq = P.qs + bid;
    uint32_t* myring = P.rings + (size_t)bid * (cap_mask + 1);

    if (t == 0) {
        for (int i = 0; i < 8; ++i) bs.ctrl[i] = 0;
        bs.misc[0] = kNoTask;
        bs.misc[1] = kNoTask;
        bs.misc[2] = __ldcg(&myq->tail0);
        bs.ctrl[6] = (int)bs.misc[2];   // count upper bound (reset leaves count == tail0)
        bs.ctrl[7] = 0;                 // head lower bound
    }
    __syncthreads();

    unsigned long long st_tasks = 0, st_pops = 0, st_sa = 0, st_steals = 0, st_idle = 0, st_pushes = 0, st_pushed = 0,
                       st_spawned = 0;
    uint64_t rng = P.seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(bid + 1)) ^ (0x9E3779B97F4A7C15ull * (uint64_t)(lane + 1));
    const uint64_t deadline = global_ns() + P.timeout_ns;
    int backoff = 32;
    int ftop = 0;
    const int fhigh = (int)P.maxspawn + 2 * kChunk;

    // per-phase clock accounting (thread 0): acquire, body, post-step, idle
    unsigned long long cy_acq = 0, cy_body = 0, cy_post = 0, cy_idle = 0;
    long long tb0 = clock64();
    for (uint32_t iter = 0;; ++iter) {
        if (warp == 0) {
            uint32_t task = kNoTask;
            int state = 0;
            if (lane == 0) {
                if ((iter & 15u) == 0u && abort_requested(P, (iter & 255u) == 0u)) {
                    state = 2;
                } else if (bs.misc[1] != kNoTask) {
                    task = bs.misc[1];   // the task retained from the previous step
                    bs.misc[1] = kNoTask;
                } else if (bs.ctrl[6] > 0) {
                    // single-task pop from the owner end; ctrl[6] is the owner's upper bound of count
                    int old = bs.ctrl[6];
                    for (int it = 0; it < 64 && old > 0; ++it) {
                        const int got = atom_cas_acq_i32(&myq->count, old, old - 1);
                        if (got == old) {
                            const uint32_t tl = bs.misc[2] - 1u;
                            bs.misc[2] = tl;
                            task = __ldcg(&myring[tl & cap_mask]);
                            ++st_pops;
                            old -= 1;
                            break;
                        }
                        old = got;
                    }
                    bs.ctrl[6] = max(old, 0);
                }
            }
            state = __shfl_sync(0xffffffffu, state, 0);
            task = __shfl_sync(0xffffffffu, task, 0);
            // Steal: warp 0 probes kProbes random victim blocks at once and claims from the
            // fullest; it keeps one task for this step and moves the rest of its claim
            // into its own deque (so the work spreads further by stealing from it).
            if (state == 0 && task == kNoTask && P.n_workers > 1) {
                constexpr int kProbes = 16;
                ++st_sa;
                int c = -1, victim = 0;
                if (lane < kProbes) {
                    rng ^= rng >> 12; rng ^= rng << 25; rng ^= rng >> 27;
                    const uint64_t r = rng * 2685821657736338717ull;
                    victim = (int)(((r >> 32) * (unsigned long long)(P.n_workers - 1)) >> 32);
                    if (victim >= bid) ++victim;
                    c = ld_cg_i32(&P.qs[victim].count);
                }
                int best = c, bl = lane;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int oc = __shfl_down_sync(0xffffffffu, best, o);
                    const int ol = __shfl_down_sync(0xffffffffu, bl, o);
                    if (oc > best) { best = oc; bl = ol; }
                }
                best = __shfl_sync(0xffffffffu, best, 0);
                bl = __shfl_sync(0xffffffffu, bl, 0);
                victim = __shfl_sync(0xffffffffu, victim, bl);
                if (best > 0) {
                    QState* vq = P.qs + victim;
                    int claim = 0;
                    uint32_t hd = 0;
                    if (lane == 0 && atom_cas_acq_i32(&vq->lock, 0, 1) == 0) {  // try-lock
                        int old = best;
                        for (int it = 0; it < 64 && old > 0; ++it) {
                            const int want = (P.steal_policy & GTAP_STEAL_ONE) ? 1 : min(16, (old + 1) >> 1);
                            const int got = atom_cas_acq_i32(&vq->count, old, old - want);
                            if (got == old) { claim = want; break; }
                            old = got;
                        }
                        if (claim > 0) hd = __ldcg(&vq->head);
                        else st_release_i32(&vq->lock, 0);
                    }
                    claim = __shfl_sync(0xffffffffu, claim, 0);
                    if (claim > 0) {
                        hd = __shfl_sync(0xffffffffu, hd, 0);
                        uint32_t v = kNoTask;
                        if (lane < claim) v = __ldcg(&P.rings[(size_t)victim * (cap_mask + 1) + ((hd + (uint32_t)lane) & cap_mask)]);
                        const uint32_t used = __reduce_or_sync(0xffffffffu, lane < claim ? v : 0u);
                        uint32_t zero;
                        asm volatile("and.b32 %0, %1, 0;" : "=r"(zero) : "r"(used));
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) {
                            __stcg(&vq->head, hd + (uint32_t)claim + zero);
                            st_release_i32(&vq->lock, 0);
                        }
                        task = __shfl_sync(0xffffffffu, v, 0);
                        ++st_steals;
                        if (claim > 1) {
                            // the own deque is empty here (the pop failed); check room anyway
                            const uint32_t tl = bs.misc[2];
                            int room = 1;
                            if (lane == 0 && tl - (uint32_t)bs.ctrl[7] + (uint32_t)(claim - 1) > cap_mask + 1) {
                                const uint32_t h2 = __ldcg(&myq->head);
                                bs.ctrl[7] = (int)h2;
                                if (tl - h2 + (uint32_t)(claim - 1) > cap_mask + 1) room = 0;
                            }
                            room = __shfl_sync(0xffffffffu, room, 0);
                            if (!room) {
                                if (lane == 0) raise_error(P, GTAP_ERR_DEQUE_OVERFLOW, -1, bid, cap_mask + 1);
                                state = 2;
                            } else {
                                if (lane >= 1 && lane < claim) __stcg(&myring[(tl + (uint32_t)(lane - 1)) & cap_mask], v);
                                __threadfence();
                                __syncwarp();
                                if (lane == 0) {
                                    bs.misc[2] = tl + (uint32_t)(claim - 1);
                                    bs.ctrl[6] += claim - 1;
                                    atomicAdd(&myq->count, claim - 1);
                                }
                            }
                        }
                    }
                }
            }
            if (state == 0 && task == kNoTask) {
                int st = 0;
                if (lane == 0) {
                    ++st_idle;
                    if ((st_idle & 3ull) == 1ull) {
                        if (ld_cg64(&P.ctl->roots_remaining.v) == 0ull) st = 2;
                        else if (global_ns() > deadline) { raise_error(P, GTAP_ERR_TIMEOUT, -1, bid, P.timeout_ns); st = 2; }
                        else if ((st_idle & 127ull) == 1ull && abort_requested(P, true)) st = 2;
                    }
                }
                state = __shfl_sync(0xffffffffu, st, 0);
            } else if (task != kNoTask && state != 2) {
                state = 1;
            }
            if (state == 1) {
                ftop = pool_refill(P, bs.fstack, ftop, (int)P.maxspawn);
                // the task's header and payload in one burst: lane i copies record bytes 16i..16i+15
                const int nrec = min(8, (int)(P.frame_bytes / 16));
                if (lane < nrec) bs.rec[lane] = __ldcg(reinterpret_cast<const uint4*>(frame_ptr(P, task)) + lane);
                if (lane == 0) {
                    if (P.fstate != nullptr) {
                        unsigned st = (task < P.n_frames) ? atomicCAS(&P.fstate[task], 3u, 1u) : 99u;  // roots start queued
                        if (st != 3u && st != 1u)
                            raise_error(P, GTAP_ERR_TASK_FAILED, (int)st, bid, (DBG_EXEC_NOT_ALLOCATED << 32) | task);
                    }
                    bs.misc[0] = task;
                    bs.ctrl[0] = ftop;
                    bs.ctrl[2] = 0;
                    bs.ctrl[4] = 0;
                    bs.ctrl[5] = 0;
                }
                backoff = 32;
            } else if (state == 0) {
                if (lane == 0) __nanosleep(backoff);
                backoff = min(backoff * 2, 1024);
            }
            if (lane == 0) bs.ctrl[3] = state;
            __syncwarp();
        }
        __syncthreads();
        const int state = bs.ctrl[3];
        if (t == 0) {
            const long long tn = clock64();
            if (state == 1) cy_acq += (unsigned long long)(tn - tb0); else cy_idle += (unsigned long long)(tn - tb0);
            tb0 = tn;
        }
        if (state == 2) break;
        if (state == 1) {
            BTaskCtx c(P, bs, bid);
            Dispatch::run(c);
        }
        __syncthreads();
        if (t == 0 && state == 1) { const long long tn = clock64(); cy_body += (unsigned long long)(tn - tb0); tb0 = tn; }
        if (warp == 0 && state == 1) {
            ++st_tasks;
            if (lane == 0) {
                const uint32_t self = bs.misc[0];
                const FrameHdr h = *bs.hdr;
                char* f = frame_ptr(P, self);
                const int jp = bs.ctrl[4];
                st_spawned += (unsigned long long)bs.ctrl[2];
                if (jp) {
                    // waiting-child count stored before any child is published
                    int k = bs.ctrl[2];
                    uint32_t w0 = (h.w0 & ~0xFF00u) | ((uint32_t)(jp - 1) << 8);
                    __stcg(reinterpret_cast<uint2*>(f), make_uint2(w0, (uint32_t)k));
                    if (k == 0) bs.staged_id[bs.ctrl[2]++] = self;
                }
                if (bs.ctrl[5]) {
                    __threadfence();
                    if (h.parent & kRootBit) {
                        RootEntry* r = &P.roots[h.parent & ~kRootBit];
                        atomicExch(&r->done, 1u);
                        atomicAdd(&P.ctl->roots_remaining.v, ~0ull);
                    } else {
                        uint32_t old = atom_add_acqrel_u32(frame_ptr(P, h.parent) + 4, 0xFFFFFFFFu);
                        if ((old & 0xFFFFFFu) == 1u) bs.staged_id[bs.ctrl[2]++] = h.parent;
                    }
                    dbg_transition(P, self, 1u, 0u, DBG_DOUBLE_FREE, (int)(h.w0 & 0xFF), bid);
                    int top = max(bs.ctrl[0], 0);
                    if (top < bs.fcap) { bs.fstack[top] = self; bs.ctrl[0] = top + 1; }
                }
            }
            __syncwarp();
            ftop = pool_spill(P, bs.fstack, max(bs.ctrl[0], 0), fhigh);
            // retain the first staged task, push the rest (one fence, one count update)
            const int nst = bs.ctrl[2];
            if (nst > 0) {
                const int npush = nst - 1;
                int overflow = 0;
                uint32_t tl = bs.misc[2];
                if (npush > 0 && lane == 0 && tl - (uint32_t)bs.ctrl[7] + (uint32_t)npush > cap_mask + 1) {
                    const uint32_t hd = __ldcg(&myq->head);
                    bs.ctrl[7] = (int)hd;
                    if (tl - hd + (uint32_t)npush > cap_mask + 1) overflow = 1;
                }
                if (__shfl_sync(0xffffffffu, overflow, 0)) {
                    if (lane == 0) raise_error(P, GTAP_ERR_DEQUE_OVERFLOW, -1, bid, cap_mask + 1);
                } else {
                    for (int i = lane; i < npush; i += 32) __stcg(&myring[(tl + (uint32_t)i) & cap_mask], bs.staged_id[1 + i]);
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) {
                        bs.misc[1] = bs.staged_id[0];
                        if (npush > 0) {
                            bs.misc[2] = tl + (uint32_t)npush;
                            bs.ctrl[6] += npush;
                            atomicAdd(&myq->count, npush);
                            ++st_pushes;
                            st_pushed += npush;
                        }
                    }
                }
            }
            __syncwarp();
            if (t == 0) { const long long tn = clock64(); cy_post += (unsigned long long)(tn - tb0); tb0 = tn; }
        }
    }
    if (t == 0) {
        WorkerStats s;
        s.tasks = st_tasks; s.steps = st_tasks; s.pops = st_pops; s.popped = st_pops;
        s.steal_attempts = st_sa; s.steals = st_steals; s.stolen = st_steals; s.idle = st_idle;
        s.pushes = st_pushes; s.pushed = st_pushed; s.spawned = st_spawned;
        s.pad[0] = cy_acq; s.pad[1] = 0; s.pad[2] = cy_body; s.pad[3] = cy_post; s.pad[4] = cy_idle;
        P.stats[bid] = s;
    }
}

}  // namespace gtap
