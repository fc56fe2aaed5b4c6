// Layout shared by the host runtime (capi.cu) and the device runtime.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define GTAP_HD __host__ __device__
#else
#define GTAP_HD
#endif

namespace gtap {

constexpr int kWarp = 32;
constexpr int kMaxQueues = 8;          // DAQ queues per warp
constexpr int kChunk = 32;             // frame IDs moved per pool chunk
constexpr uint32_t kRootBit = 0x80000000u;
constexpr uint32_t kNoTask = 0xFFFFFFFFu;
constexpr int kRootArgBytes = 64;      // per-root argument block
constexpr int kHdrBytes = 16;

// Built-in program type IDs (frame header "type" field).  0 is never a valid type.
enum ProgType : int {
    T_NONE = 0,
    // thread mode
    T_FIB = 1,
    T_NQUEENS = 2,
    T_UTS = 3,
    T_UTS_RANGE = 4,     // spawns a contiguous range of a node's children
    T_INTEGRATE = 5,
    T_KCLIQUE_ROOT = 6,  // range of DAG edges
    T_KCLIQUE_EDGE = 7,  // one edge / a sub-range of a candidate set
    T_KCLIQUE_SET = 8,
    T_BINTREE = 9,       // full binary tree microbenchmark (Sec. 6.1, 6.2)
    T_TSORT = 10,        // thread-mode Cilksort: sort a range
    T_TMERGE = 11,       // thread-mode Cilksort: merge two runs
    T_KCLIQUE_PIV = 12,  // k-clique by pivoting: branch range of a bitset-encoded candidate subgraph
    T_KCLIQUE_PIVB = 13, // k-clique by pivoting: a node of a candidate subgraph of more than 64 vertices
    // block mode
    T_MSORT = 16,
    T_MMERGE = 17,
    T_INTEGRATE_BLK = 18,
    T_DTT = 19,
    T_BINTREE_BLK = 20,
    T_MAX = 32
};

// Program-set bits selecting a kernel instantiation (which state machines are compiled in).
enum ProgSet : unsigned {
    PS_FIB = 1u << 0,
    PS_NQUEENS = 1u << 1,
    PS_UTS = 1u << 2,
    PS_INTEGRATE = 1u << 3,
    PS_KCLIQUE = 1u << 4,
    PS_BINTREE = 1u << 5,
    PS_CILKSORT = 1u << 6,
    PS_THREAD_ALL = PS_FIB | PS_NQUEENS | PS_UTS | PS_INTEGRATE | PS_KCLIQUE | PS_BINTREE | PS_CILKSORT,
    PS_MSORT = 1u << 8,
    PS_INTEGRATE_BLK = 1u << 9,
    PS_DTT = 1u << 10,
    PS_BINTREE_BLK = 1u << 11,
};

// Thread-mode queue management (gtap_config.scheduler; Sec. 6.5).
enum Sched : int { SCHED_BATCHED = 0, SCHED_GLOBAL = 1, SCHED_SINGLE = 2 };

constexpr uint64_t kScratchBlock = 4096;   // bytes per recycled scratch block
constexpr uint64_t kScratchLargeBlocks = 16; // blocks per recycled large chunk (64 KiB)

// Frame header flag bits.
constexpr uint32_t kFlagAccumulate = 1u;  // child result is added (u64) into the parent slot

// Task record header, 16 bytes, at the start of every frame.
//   w0      = type:8 | pc:8 | flags:8 | unused:8
//   pending = outstanding children:24 | continuation queue:8
//   parent  = parent task ID, or kRootBit | root index
//   w3      = slot:16 (byte offset / 8 of the result slot in the parent record) | aux:16
struct FrameHdr {
    uint32_t w0;
    uint32_t pending;
    uint32_t parent;
    uint32_t w3;
};

// Per-queue shared state, 16 bytes.  head and count are the thief-visible
// words (Sec. 5.1.3); tail0 hands the owner its initial tail (the live tail is
// kept in shared memory by the owner).
struct QState {
    int count;
    uint32_t head;
    int lock;
    uint32_t tail0;
};

struct ErrorRecord {
    int code;
    int task_type;
    int worker;
    int pad;
    unsigned long long detail;
};

// Control block.  Hot words sit on their own 128-byte lines.
struct alignas(128) Line128 { unsigned long long v; char pad[120]; };
struct DevControl {
    Line128 roots_remaining;   // decremented when a root completes (termination)
    Line128 abort_flag;        // nonzero: every worker drains and exits
    Line128 bump;              // next never-used frame ID
    Line128 cq_enq;            // chunk-queue enqueue ticket
    Line128 cq_deq;            // chunk-queue dequeue ticket
    Line128 scratch_top;       // bytes taken from the scratch arena
    Line128 inflight;          // serving: roots admitted and not yet completed
    Line128 cq_avail;          // chunks whose enqueue has completed and that no dequeuer reserved
    Line128 sc_enq, sc_deq, sc_avail;   // scratch free-block queue tickets / completed frees
    Line128 lc_enq, lc_deq, lc_avail;   // the same for recycled large chunks (kScratchLargeBlocks blocks each)
    Line128 out_tail;          // serving: completions written to the outbox
    Line128 admitted;          // serving: requests admitted so far
    Line128 gq_enq, gq_deq, gq_avail;   // central-queue scheduler: tickets and completed publications
    alignas(128) ErrorRecord err;
};

// Serving: a root slot whose `done` word holds this value is free for a new request.
constexpr unsigned int kRootSlotFree = 0xFFFFFFFFu;

struct RootEntry {
    unsigned long long result[2];
    unsigned int done;
    unsigned int type;
    unsigned long long req;    // serving: the request's sequence number
};

// Serving (resident kernel).  The host writes requests into a ring of inbox
// slots in mapped pinned memory and reads completions from a ring of outbox
// entries there; both rings are indexed by monotonically increasing sequence
// numbers, and a slot is valid when its seq field equals its sequence + 1.
struct InboxSlot {
    unsigned long long seq;
    uint32_t type;
    uint32_t queue;
    unsigned char payload[48];
    unsigned char env[64];
};
struct OutboxEntry {
    unsigned long long seq;
    unsigned long long req;
    unsigned long long result[2];
    int status;
    int pad[3];
};
struct HostFlags {            // mapped pinned host memory
    int abort;                // same role as host_abort in batch runs
    int dev_error;            // device: first error code of the session (0 = none)
    unsigned long long shutdown;        // host: no more requests; drain and exit
    unsigned long long inbox_consumed;  // device: requests taken from the inbox
    unsigned long long out_consumed;    // host: completions read from the outbox
};

// A root as queued by the host: its initial record payload and a read-only
// per-root environment (e.g. the device buffers a program works on).
constexpr int kRootPayloadBytes = 48;
struct RootDesc {
    uint32_t type;
    uint32_t queue;
    uint32_t flags;
    uint32_t pad;
    unsigned char payload[kRootPayloadBytes];
    unsigned char env[kRootArgBytes];
};

struct WorkerStats {
    unsigned long long tasks, steps, pops, popped, steal_attempts, steals, stolen, idle, pushes, pushed, spawned;
    unsigned long long pad[5];   // thread mode: SM cycles spent in pop, steal, execute, retain/push, idle
};

// Kernel parameters (passed by value).
struct KParams {
    char* frames;
    uint64_t n_frames;
    uint32_t frame_bytes;
    uint32_t n_workers;       // warps (thread mode) or blocks (block mode)
    uint32_t n_queues;        // per worker
    uint32_t ring_mask;       // ring capacity - 1 (power of two)
    uint32_t* rings;          // [n_workers * n_queues][capacity]
    QState* qs;               // [n_workers * n_queues]
    unsigned long long* cq_seq;  // chunk queue sequence numbers [ncq]
    uint32_t* cq_ids;         // [ncq][kChunk]
    uint64_t ncq_mask;
    DevControl* ctl;
    RootEntry* roots;
    const RootDesc* root_desc;
    uint32_t n_roots;
    uint32_t maxspawn;        // max children one step stages: per lane (thread mode) / per block (block mode)
    uint32_t warp_smem;       // thread mode: shared bytes per warp (runtime part + the program set's warp area)
    WorkerStats* stats;
    volatile int* host_abort; // mapped pinned host word, may be null
    uint64_t timeout_ns;
    uint64_t seed;
    int steal_policy;
    int idle_backoff_ns;      // thread mode: longest sleep of an idle warp between steal rounds
    int pad0;
    char* scratch;            // scratch blocks for programs (k-clique candidate sets), kScratchBlock bytes each
    uint64_t scratch_bytes;   // bytes of the block region
    unsigned long long* sq_seq;   // free-block queue: sequence numbers and block ids
    uint32_t* sq_ids;
    uint64_t sq_mask;
    unsigned long long* lq_seq;   // free large-chunk queue: sequence numbers and first-block ids
    uint32_t* lq_ids;
    uint64_t lq_mask;
    // serving mode (resident kernel)
    int serving;
    uint32_t inbox_cap, outbox_cap;
    int pad1;
    InboxSlot* inbox;          // mapped pinned host memory (device pointers)
    OutboxEntry* outbox;
    HostFlags* hflags;
    unsigned long long admit_reserve;   // admit a request only while at least this many records are free
    unsigned int* fstate;     // debug: per-record state (0 free, 1 allocated, 2 running, 3 queued), or null
    unsigned long long* flog; // debug: last 8 events per record
    unsigned int* flogn;      // debug: event count per record
    // central-queue scheduler (GTAP_SCHED_GLOBAL): slot words (sequence:32 | task id:32)
    unsigned long long* gq;
    uint64_t gq_mask;
};

// Debug-check failure codes (error detail = code << 32 | record id).
enum DebugFault : unsigned long long {
    DBG_DOUBLE_ALLOC = 1, DBG_DOUBLE_FREE = 2, DBG_EXEC_NOT_ALLOCATED = 3, DBG_BAD_ID = 4,
};

// Shared-memory sizing (thread mode: per warp; block mode: per block, runtime part).
GTAP_HD constexpr int thread_fcap(int maxspawn) { return 32 * maxspawn + 3 * kChunk + 32; }
GTAP_HD constexpr int thread_scap(int maxspawn) { return 32 * (maxspawn > 1 ? maxspawn : 1); }
GTAP_HD constexpr int thread_warp_smem(int maxspawn) {
    return 256 /*ctrl, cls_count, tail, push_off, hint, head_lb*/ + 128 + 128 +
           4 * thread_fcap(maxspawn) + 4 * thread_scap(maxspawn) + ((thread_scap(maxspawn) + 15) / 16) * 16;
}

// Block mode: step_max = most children one block step can spawn (all threads together).
GTAP_HD constexpr int block_fcap(int step_max) { return step_max + 3 * kChunk + 32; }
GTAP_HD constexpr int block_scap(int step_max) { return ((step_max + 2 + 3) / 4) * 4; }
GTAP_HD constexpr int block_rt_smem(int step_max) { return 192 + 4 * block_fcap(step_max) + 4 * block_scap(step_max); }

}  // namespace gtap
