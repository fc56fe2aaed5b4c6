/*
 * gtap.h -- C ABI of a GPU-resident fork-join task runtime for GB300 (sm_103a).
 *
 * The runtime executes fine-grained fork-join task programs inside one
 * persistent kernel: every warp (thread mode) or thread block (block mode)
 * owns a deque of runnable task IDs, acquires work by batched pop and random
 * work stealing, suspends a task at a join by storing its resume point in the
 * task record, and re-enqueues it in place when its last child completes
 * (paper Sec. 5.1; Algorithms 1 and 2).  Divergence-Aware Queueing (DAQ)
 * gives each warp several queues and fills a warp batch from one queue
 * (Sec. 4.2).  Task programs are built-in continuation state machines; they
 * are selected by name with gtap_register_task.
 *
 * Conventions for every call:
 *   - Every function returns a gtap_status; nothing throws or aborts the
 *     process.  GTAP_OK is 0.
 *   - Pointers documented as "device" must be device-accessible memory of
 *     the current CUDA device (e.g. cudaMalloc or a torch CUDA tensor); all
 *     others are host memory.  Device buffers passed in program arguments are
 *     owned by the caller and must stay alive until gtap_wait returns.
 *   - A context is used by one host thread at a time.
 *
 * Storage (Sec. 4: everything is preallocated before a run, no device-side
 * allocation during it): gtap_init allocates the task-record pool, the
 * deques and the control block with cudaMalloc (or carves them from a
 * caller-provided device arena) and gtap_finalize releases them.
 */
#ifndef GTAP_H_
#define GTAP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes.  Device-side failures (capacity exhaustion, Sec. 4: "aborts
 * execution with a structured error report") are reported by gtap_wait and
 * detailed by gtap_last_error. */
typedef enum {
    GTAP_OK = 0,
    GTAP_ERR_INVALID_ARG = 1,     /* bad argument, unknown program name or handle */
    GTAP_ERR_NO_MEMORY = 2,       /* host or device allocation failed at init */
    GTAP_ERR_POOL_EXHAUSTED = 3,  /* task-record pool ran out during a run */
    GTAP_ERR_DEQUE_OVERFLOW = 4,  /* a push found its deque full */
    GTAP_ERR_LIST_OVERFLOW = 5,   /* a fixed-capacity output list (FMM interaction lists) overflowed */
    GTAP_ERR_TIMEOUT = 6,         /* run deadline or gtap_wait timeout reached; the kernel was told to stop */
    GTAP_ERR_CUDA = 7,            /* a CUDA runtime call failed */
    GTAP_ERR_BUSY = 8,            /* a run is in flight (call gtap_wait first) */
    GTAP_ERR_UNKNOWN_TASK = 9,    /* a task record carried an unregistered type */
    GTAP_ERR_TASK_FAILED = 10,    /* a task program reported failure (e.g. scratch arena exhausted) */
    GTAP_ERR_NOT_READY = 11       /* the requested result is not available yet */
} gtap_status;

typedef enum { GTAP_MODE_THREAD = 0, GTAP_MODE_BLOCK = 1 } gtap_mode;

/* Steal policy bits (gtap_config.steal_policy). */
#define GTAP_STEAL_FILL 0      /* steal whenever the warp batch is not full (Alg. 1) */
#define GTAP_STEAL_EMPTY 1     /* steal only when the warp has no task at all */
#define GTAP_STEAL_HALF 2      /* thread mode: claim at most half of the victim's queue (else up to 32 - cnt) */
#define GTAP_STEAL_ONE 4       /* block mode: steal exactly one task (else up to half of the victim's queue,
                                  at most 16: one runs now, the rest move to the thief's own deque) */

/* Optional configuration; a zero field selects the default.  Pass NULL for
 * all defaults. */
typedef struct {
    int blocks_per_sm;      /* persistent grid = blocks_per_sm x SM count (default: 4 thread mode, 2 block mode) */
    int threads_per_block;  /* thread mode: 32..256, multiple of 32 (default 256); block mode: 128 or 256
                               (default 256), or 32 for "bintree_block" */
    int deque_capacity;     /* ring slots per queue, power of two (default 4096 thread mode, 1024 block mode) */
    int steal_policy;       /* GTAP_STEAL_* bits (default GTAP_STEAL_FILL) */
    int max_roots;          /* capacity of the root table (default 4096) */
    int frame_bytes;        /* thread-mode task-record size, 64 or 128 (default 64) */
    void* device_arena;     /* optional caller-owned device memory used for all runtime storage */
    size_t arena_bytes;     /* its size; gtap_init fails with GTAP_ERR_NO_MEMORY if too small */
    void* stream;           /* cudaStream_t for runs (default: the legacy default stream) */
    uint64_t timeout_ns;    /* device-side run deadline (default 60 s); exceeded -> GTAP_ERR_TIMEOUT */
    uint64_t seed;          /* victim-selection seed (default 0x5EED) */
    size_t scratch_bytes;   /* device scratch arena for programs that need it (k-clique candidate sets and
                               pivoting rows): 4 KiB blocks and 64 KiB chunks, each size recycled through
                               its own free queue, default 0 */
    int grid_blocks;        /* explicit persistent grid size (overrides blocks_per_sm x SM count), e.g. 1 */
    int debug_checks;       /* 1: track every record's state (free / allocated / running) and report
                               double allocation, double free or double execution as GTAP_ERR_TASK_FAILED */
    int scheduler;          /* thread-mode queue management (GTAP_SCHED_*, default GTAP_SCHED_BATCHED);
                               the alternatives exist for the scheduler comparison of Sec. 6.5 */
    int idle_backoff_ns;    /* thread mode: longest sleep of an idle warp between steal rounds, 32..65536 ns
                               (default 512); longer relieves L2 of idle probing, shorter spreads new work faster */
} gtap_config;

/* Thread-mode scheduler designs compared in Sec. 6.5 ("GPU-Side Scheduler
 * Comparison").  All share the runtime (records, joins, termination) and
 * differ only in queue management.
 *   GTAP_SCHED_BATCHED: per-warp deques with warp-cooperative batched pop and
 *     steal (Alg. 1 and 2), the default.
 *   GTAP_SCHED_GLOBAL: one centralised queue shared by every warp: a warp
 *     claims up to 32 - cnt tasks per claim from its head and publishes new
 *     tasks at its tail (ticketed slots, one claim and one publish per batch).
 *   GTAP_SCHED_SINGLE: per-warp deques, non-batched: the warp's lanes issue
 *     up to 32 single-task pops, then single-task steals, one CAS per task. */
#define GTAP_SCHED_BATCHED 0
#define GTAP_SCHED_GLOBAL 1
#define GTAP_SCHED_SINGLE 2

/* Per-run statistics, summed over workers (gtap_get_stats). */
typedef struct {
    uint64_t tasks_executed;     /* task steps executed (a suspended task that resumes counts twice) */
    uint64_t tasks_created;      /* tasks spawned in the run, roots included */
    uint64_t steps;              /* scheduler iterations that executed at least one task */
    uint64_t pops, popped;       /* successful pop claims and tasks they returned */
    uint64_t steal_attempts, steals, stolen;
    uint64_t idle_iterations;
    uint64_t pushes, pushed;     /* push batches and tasks they published */
    uint64_t frames_high_water;  /* fresh records ever taken from the pool (bump pointer) */
    uint64_t scratch_used;       /* bytes taken from the scratch arena */
    int n_workers;               /* warps (thread mode) or blocks (block mode) in the grid */
    int grid_blocks, threads_per_block;
    float kernel_ms;             /* duration of the last persistent kernel (CUDA events on its stream) */
    float run_ms;                /* the whole last run: root upload + reset kernel + persistent kernel */
    uint64_t cycles_pop, cycles_steal, cycles_exec, cycles_push, cycles_idle;  /* SM cycles per scheduler
                                    phase summed over workers (tracing counters); block mode reports
                                    acquire in cycles_pop, task bodies in cycles_exec, the post-step in
                                    cycles_push and cycles_steal = 0 */
} gtap_stats;

/* Structured error report (Sec. 4: capacity exhaustion aborts with a report). */
typedef struct {
    int code;        /* gtap_status of the first device-side error, 0 if none */
    int task_type;   /* type of the task that hit it, -1 if not task-specific */
    int worker;      /* warp or block index */
    int pad;
    uint64_t detail; /* e.g. the capacity that was exceeded */
} gtap_error_info;

typedef struct gtap_ctx gtap_ctx;

/* Create a context (Sec. 4, gtap_initialize(config): all runtime storage
 * is reserved before any task runs): mode, number of DAQ queues per warp
 * (1..8; block mode requires 1, as the queue clause is not supported there,
 * Sec. 4.3), and the size of the task-record pool in bytes.  All storage is
 * allocated here, or carved from cfg->device_arena when the caller gives one
 * (see gtap_arena_bytes for the size it needs).
 * Errors: GTAP_ERR_INVALID_ARG, GTAP_ERR_NO_MEMORY, GTAP_ERR_CUDA. */
gtap_status gtap_init(gtap_mode mode, int n_queues, size_t frame_pool_bytes, const gtap_config* cfg,
                      gtap_ctx** out);

/* Bytes of device memory gtap_init needs for these arguments: the size a
 * caller-owned cfg->device_arena must have (256-byte aligned).  Reads the
 * SM count of the current device; allocates nothing.
 * Errors: those of gtap_init's argument checks, GTAP_ERR_CUDA. */
gtap_status gtap_arena_bytes(gtap_mode mode, int n_queues, size_t frame_pool_bytes, const gtap_config* cfg,
                             size_t* out);

/* Select a built-in task program by name and get its type ID for
 * gtap_spawn_root (the programs of Sec. 6, written as the continuation state
 * machines Sec. 5.2 lowers tasks into).  Thread mode: "fib", "nqueens", "uts",
 * "kclique", "integrate", "bintree", "cilksort".  Block mode: "mergesort",
 * "integrate_block", "fmm_dtt", "bintree_block".
 * Errors: GTAP_ERR_INVALID_ARG for an unknown name or the wrong mode. */
gtap_status gtap_register_task(gtap_ctx* ctx, const char* program, int* out_type);

/* Queue a root task for the next gtap_run: its arguments (the program's
 * gtap_*_args struct) are copied now (firstprivate, Sec. 4.1).  queue
 * selects the DAQ queue of the root.  Roots of one run are spread over the
 * workers round-robin, so many instances of uneven size run in one launch.
 * out_handle identifies the root for gtap_read_result.
 * Errors: GTAP_ERR_INVALID_ARG (unregistered type, args too large, table full), GTAP_ERR_BUSY. */
gtap_status gtap_spawn_root(gtap_ctx* ctx, int type, const void* args, size_t args_bytes, int queue,
                            uint64_t* out_handle);

/* Start one persistent-kernel run over the queued roots (Sec. 4,
 * gtap_launch; the kernel is the scheduler loop of Alg. 1), asynchronously on
 * the configured stream: a reset kernel re-zeroes deques, pool and control
 * words and writes the root records, then the scheduler kernel runs until
 * every root has completed (or an error/abort).  The queued roots stay
 * queued, so calling gtap_run again re-runs the same roots.
 * Errors: GTAP_ERR_INVALID_ARG (no roots), GTAP_ERR_BUSY, GTAP_ERR_CUDA. */
gtap_status gtap_run(gtap_ctx* ctx);

/* Wait for the run started by gtap_run (Sec. 4: the host regains control
 * when every task has completed, Alg. 1's termination test), at most
 * timeout_ms milliseconds (0 = the config's device deadline plus a margin).  Never hangs: on
 * timeout it raises the device abort flag, waits for the kernel to drain and
 * returns GTAP_ERR_TIMEOUT.  Returns the device-side error code if the run
 * failed.  Results and statistics are read back here. */
gtap_status gtap_wait(gtap_ctx* ctx, uint64_t timeout_ms);

/* Copy the result of a completed root (bytes <= 16) into out (host): the
 * value the root task returned (Sec. 4.1, values returned from tasks; Sec.
 * 5.1.2, the result a completing task writes for its parent).
 * Errors: GTAP_ERR_INVALID_ARG (bad handle), GTAP_ERR_NOT_READY. */
gtap_status gtap_read_result(gtap_ctx* ctx, uint64_t handle, void* out, size_t bytes);

/* Statistics of the last completed run: task, pop, steal and push counts
 * of the scheduler loop (Alg. 1, Alg. 2) and its per-phase cycle counters. */
gtap_status gtap_get_stats(gtap_ctx* ctx, gtap_stats* out);

/* Structured report of the last device-side error (code 0 if none). */
gtap_status gtap_last_error(gtap_ctx* ctx, gtap_error_info* out);

/* Forget the queued roots (the next gtap_spawn_root starts a new batch). */

/* Change the device-side run deadline (gtap_config.timeout_ns) of later runs;
 * 0 restores the default of 60 s.  A run past its deadline drains and
 * gtap_wait returns GTAP_ERR_TIMEOUT (Sec. 4: execution aborts with a
 * structured report).  Drops a captured graph.  Errors: GTAP_ERR_BUSY while a
 * run is in flight. */
gtap_status gtap_set_timeout(gtap_ctx* ctx, uint64_t timeout_ns);
gtap_status gtap_clear_roots(gtap_ctx* ctx);

/* ------------------------------------------------------------------------
 * Serving: a resident persistent kernel fed through a host-to-device inbox
 * (thread mode).  gtap_serve_start launches the scheduler kernel, which keeps
 * running; gtap_submit queues a request (a root of a registered program, its
 * arguments copied now) in a ring of mapped pinned host memory; a device warp
 * admits it once enough task records are free (at least 1/64 of the pool) and
 * a root slot and an outbox entry are available, so requests that arrive while
 * others run start as soon as memory frees up and their work overlaps on the
 * device; each completion is written to a mapped outbox that gtap_poll reads.
 * Between gtap_serve_start and gtap_serve_stop no gtap_run is allowed. */
typedef struct {
    uint64_t req;        /* the id gtap_submit returned */
    uint64_t result[2];  /* the root's result (as gtap_read_result would return it) */
    int32_t status;      /* 0 */
    int32_t pad;
} gtap_completion;

/* Launch the resident kernel.  Errors: GTAP_ERR_INVALID_ARG (block mode or no
 * registered program), GTAP_ERR_BUSY, GTAP_ERR_NO_MEMORY, GTAP_ERR_CUDA. */
gtap_status gtap_serve_start(gtap_ctx* ctx);

/* Queue one request; never blocks.  Returns GTAP_ERR_BUSY when the inbox ring
 * (max_roots slots) is full, GTAP_ERR_INVALID_ARG for bad arguments. */
gtap_status gtap_submit(gtap_ctx* ctx, int type, const void* args, size_t args_bytes, int queue, uint64_t* out_req);

/* Copy up to max completed requests (in completion order) into out; *n gets
 * the number copied (0 if none is ready).  Also valid after gtap_serve_stop.
 * Returns the device's error code once the session has failed (the kernel then
 * drains; call gtap_serve_stop), else GTAP_OK. */
gtap_status gtap_poll(gtap_ctx* ctx, gtap_completion* out, int max, int* n);

/* Serving progress, read from host and mapped memory without touching the
 * device: up to n of [0] requests submitted, [1] requests the device has
 * admitted (taken from the inbox), [2] completions gtap_poll has returned.
 * [0] - [1] is the inbox backlog (waiting for admission), [1] - [2] the
 * requests on the device or completed and not yet polled. */
gtap_status gtap_serve_progress(gtap_ctx* ctx, uint64_t* out, int n);

/* Close the inbox: the kernel admits what was submitted, finishes it and
 * exits; waits at most timeout_ms (0: the device deadline), then raises the
 * abort word.  Returns the device status. */
gtap_status gtap_serve_stop(gtap_ctx* ctx, uint64_t timeout_ms);

/* Capture one run of the currently queued roots (root upload, reset kernel,
 * persistent kernel) as a CUDA graph; later gtap_run calls replay the graph
 * instead of issuing the steps one by one, until the queued roots change
 * (gtap_spawn_root or gtap_clear_roots drop the graph).  Capture happens on a
 * stream the context owns (capture cannot use the legacy default stream);
 * replays run there too and gtap_wait waits for them.  Batching roots plus
 * graph replay is the "many instances, one launch" form of the runtime.
 * Errors: GTAP_ERR_INVALID_ARG (no roots), GTAP_ERR_BUSY, GTAP_ERR_CUDA. */
gtap_status gtap_capture_graph(gtap_ctx* ctx);

/* Diagnostic snapshot of the device scheduler state after a run (for
 * post-mortem of an error or timeout).  Fills up to n of: [0] roots
 * remaining, [1] fresh-record bump pointer, [2] chunk-queue enqueue ticket,
 * [3] chunk-queue dequeue ticket, [4] tasks left in all deques (sum of
 * count), [5] queues with count > 0, [6] queue locks held, [7] largest count,
 * [8] abort flag.  Returns GTAP_ERR_BUSY while a run is in flight. */
gtap_status gtap_debug_snapshot(gtap_ctx* ctx, uint64_t* out, int n);

/* Human-readable name of a status code (static storage). */
const char* gtap_status_string(gtap_status s);

/* Release every resource of the context (Sec. 4, gtap_finalize; waits for
 * an in-flight run first). */
gtap_status gtap_finalize(gtap_ctx* ctx);

/* ------------------------------------------------------------------------
 * Built-in program arguments (passed to gtap_spawn_root).
 * Routing ("route") selects the program's DAQ routing function; 0 sends
 * every task to queue 0, which is the same as omitting the queue clause.
 * Any routing gives the same result (the queue clause has no effect on
 * program semantics, Sec. 4.2).
 * ---------------------------------------------------------------------- */

/* fib(n) (Sec. 6.3).  cutoff 0 (or <= 2): a task at every call.  cutoff c > 2:
 * a call with n < c is a leaf task that computes fib(n) by the serial
 * recursion in its lane (Sec. 6.3.2).  Result: int64 fib(n).
 * route 1: recursive calls -> q0, leaves -> q1, continuations -> q2 (mod n_queues). */
typedef struct { int32_t n; int32_t route; int32_t cutoff; int32_t pad; } gtap_fib_args;

/* N-Queens by bitmask backtracking (Sec. 6.3).  cutoff 0: one task per placed
 * row; cutoff d > 0: a board with d rows placed is a leaf task that finishes
 * the search serially (Sec. 6.3.1 uses d = 7).  Result: uint64 solution count.
 * route 1: queue = depth mod n_queues; route 2: recursive tasks -> q0, cutoff
 * leaves -> q1 (Sec. 6.3.2, two queues). */
typedef struct { int32_t n; int32_t route; int32_t cutoff; int32_t pad; } gtap_nqueens_args;

/* Unbalanced hashed tree: root id splitmix64(seed), root_children children at
 * the root, m children below iff splitmix64(v ^ 0xD1B54A32D192ED03) < threshold.
 * Result: uint64 nodes in the high 32 bits, leaves in the low 32 bits.
 * route 1: nodes with children -> q0, leaves -> q1, continuations -> q2. */
typedef struct { uint64_t seed; uint64_t threshold; uint32_t root_children; uint32_t m; int32_t route; int32_t pad; } gtap_uts_args;

/* Adaptive trapezoid integration of 1/(1+25x^2) over [a, b] (Program 1).
 * Thread mode ("integrate") and block mode ("integrate_block").  Result: double. */
typedef struct { double a; double b; double eps; } gtap_integrate_args;

/* Full binary task tree (Sec. 6.1 "Understanding the Execution Modes", Sec. 6.2
 * "Effect of Divergence-Aware Queueing"), thread mode ("bintree") and block
 * mode ("bintree_block").  Node ids: root 1, children of v are 2v and 2v+1;
 * the leaves are the 2^depth nodes of level `depth`.  Each leaf runs a
 * data-parallel loop of `iters` iterations of one of K (1..4) compute
 * functions, k(v) = (splitmix64(v) >> 32) mod K (0 when K = 1), known at
 * spawn:  value(v) = sum_{i < iters} g_k((v << 32) + i) mod 2^64 with
 *   g_0(x): z = x * 0x9E3779B97F4A7C15; z ^= z >> 29; z *= 0xBF58476D1CE4E5B9; z ^ (z >> 32)
 *   g_1(x): z = x ^ (x << 13); z ^= z >> 7; z ^= z << 17; z * 0x2545F4914F6CDD1D
 *   g_2(x): z = (x + 0x632BE59BD9B4E019) * 0x94D049BB133111EB; rotl(z, 23) ^ (z >> 11)
 *   g_3(x): z = x ^ (x >> 32); z *= 0xD6E8FEB86659FD93; z ^ (z >> 28)
 * Result: uint64 sum of the leaf values mod 2^64.  Thread mode: one lane runs
 * a leaf's loop; route 1 sends inner nodes to queue 0 and a leaf of function k
 * to queue 1 + k (DAQ; use n_queues = K + 1).  Block mode: the block runs a
 * leaf's loop with its iterations strided over the threads; cutoff c > 0 makes
 * a node c levels above the leaves run its whole subtree as one task (thread
 * mode requires cutoff 0).  depth <= 30. */
typedef struct { int32_t depth; int32_t iters; int32_t K; int32_t route; int32_t cutoff; int32_t pad; } gtap_bintree_args;

/* Thread-mode Cilksort ("cilksort", Sec. 6.3; Sec. 6.3.2 runs it with three
 * DAQ queues) of n < 2^32 uint32 keys from src (device, read only) into dst
 * (device); tmp (device, n keys) is scratch; src may equal dst.  A range of at
 * most sort_cutoff (<= 256, default 64) keys is a leaf task whose lane sorts it
 * alone; a larger range sorts its halves into the other buffer and then merges
 * them back.  A merge of at most merge_cutoff (default 256) outputs is a leaf
 * task merging serially; a larger merge writes the longer run's middle key x
 * to its final place and forks the merges on either side of it (the shorter
 * run cut at its first key not less than x).  route 1: recursive tasks -> q0,
 * serial sorts -> q1, serial merges -> q2.  Result: none (8 zero bytes). */
typedef struct { const uint32_t* src; uint32_t* dst; uint32_t* tmp; uint64_t n; uint32_t sort_cutoff;
                 uint32_t merge_cutoff; int32_t route; int32_t pad; } gtap_cilksort_args;

/* Block-mode mergesort (Cilksort with a forked parallel merge, Sec. 6.3) of
 * n uint32 keys from src (device, read only) into dst (device); tmp (device,
 * n keys) is scratch.  src may equal dst for an in-place sort.  Ranges of at
 * most `leaf` keys (<= 4096) are sorted by one block; merges of at most
 * `merge_cutoff` output keys are merged by one block, larger ones fork.
 * Result: none (8 zero bytes). */
typedef struct { const uint32_t* src; uint32_t* dst; uint32_t* tmp; uint64_t n; uint32_t leaf; uint32_t merge_cutoff; } gtap_mergesort_args;

/* k-clique counting by graph orientation (Sec. 6.4.2), thread mode ("kclique").
 * off/adj/src are the oriented DAG from gtap_kclique_orient (device, caller
 * owned, read only during the run).  Every DAG edge (u, v) of the root's
 * range (all edges: [0, m)) counts the
 * (k-2)-cliques of C = N+(u) n N+(v); a set larger than split_threshold
 * (<= 64, default 64) is materialised in the context's scratch arena
 * (gtap_config.scratch_bytes) and forked into child tasks over its branch
 * range; smaller ones are counted with 64-bit adjacency rows.  Where rows are
 * built (at least two more vertices to choose), the lanes of a warp that run
 * the same step process their edges or branches together, one at a time
 * (binary searches split over the lanes, C and its rows in the warp's shared
 * memory); elsewhere each lane intersects its own lists.  A first-level set is
 * written by its own task when that task starts (waiting first-level tasks
 * hold no scratch); deeper sets by the task that spawns them.
 * route 1: queue = recursion depth mod n_queues.  k in [3, 16].  Result: uint64 count.
 *
 * algorithm 1 (GTAP_KCLIQUE_PIVOT) counts by pivoting instead (Sec. 6.4.2, the
 * second algorithm): candidate sets of at most split_threshold vertices are
 * encoded as 64-bit adjacency rows in the lane and counted by a pivot search
 * (the pivot is the vertex with the most neighbours in the set, ties to the
 * lowest position; its non-neighbours and itself are the branches; an empty
 * set adds C(pivots, vertices still to choose)); sets of up to 64 vertices are
 * encoded as a bitset subgraph in the scratch arena and their branch range is
 * split over child tasks ("bitset-encoded split"); a first-level set of 65 to
 * 1024 vertices is pivoted the same way over multi-word bitset rows that its
 * own task writes into the scratch arena when it starts, and its branch sets
 * switch to the 64-bit form once they fit.  A first-level set of more than
 * 1024 vertices fails the run with GTAP_ERR_INVALID_ARG.  Same count as
 * orientation. */
#define GTAP_KCLIQUE_ORIENT 0
#define GTAP_KCLIQUE_PIVOT 1
typedef struct { const int64_t* off; const int32_t* adj; const int32_t* src;
                 int64_t edge_begin, edge_end;   /* the root counts DAG edges [edge_begin, edge_end) */
                 int32_t k; int32_t split_threshold; int32_t route; int32_t algorithm; } gtap_kclique_args;

/* Orient an undirected simple graph (each edge once, as m int32 pairs in edges,
 * device) by the order (degree, id): outputs off[n+1] (int64), adj[m] (out-lists
 * sorted by id) and src[m] (the source vertex of each DAG edge), all device and
 * caller owned.  work: device int32 scratch of at least 4*n + 16 elements.
 * Stream-ordered on stream; returns after completion.  Errors:
 * GTAP_ERR_INVALID_ARG (bad sizes, or an out-list longer than 8192). */
gtap_status gtap_kclique_orient(const int32_t* edges, int64_t m, int64_t n, int64_t* off, int32_t* adj,
                                int32_t* src, int32_t* work, void* stream);

/* Atomic-rate microbenchmark (the ceilings of the thread-mode scheduler).  kind:
 * 0 scattered acq_rel atomic add with return (the join decrement), 1 scattered
 * fire-and-forget 64-bit add (accumulating joins), 2 CAS on one word per warp
 * (deque claims), 3 CAS on one shared word (a hot word), 4 scattered L2 loads.
 * region: device buffer of region_bytes (its contents are overwritten).
 * Runs one warm-up and one timed launch of blocks x threads threads, each doing
 * iters operations (kinds 2-3: one lane per warp); *ms_out gets the timed
 * launch's duration and *ops_out the operations it performed. */
gtap_status gtap_microbench(int kind, void* region, uint64_t region_bytes, int blocks, int threads, int iters,
                            float* ms_out, double* ops_out, void* stream);

/* ------------------------------------------------------------------------
 * Autotuner.  For one program and one batch of roots, pick blocks per SM,
 * ring capacity, DAQ queue count, steal policy and (thread mode) the idle
 * back-off by coordinate descent over
 *   thread mode: blocks/SM {1,2,4,6,8}, steal {FILL, EMPTY, HALF, EMPTY|HALF},
 *                queues {1,2,3,4}, capacity {1024, 4096, 16384},
 *                idle back-off {512, 2048, 8192} ns;
 *   block mode:  blocks/SM {1,2,3,4,6}, steal {half of the victim, ONE},
 *                queues {1}, capacity {1024, 4096, 16384},
 * starting from 4 blocks/SM, capacity 4096, n_queues queues, default
 * stealing and the base configuration's back-off; tune_mask selects the
 * dimensions that may change (GTAP_TUNE_BLOCKS | GTAP_TUNE_STEAL |
 * GTAP_TUNE_QUEUES | GTAP_TUNE_CAPACITY | GTAP_TUNE_BACKOFF, 0 = all).  Each trial creates a context (gtap_init with `base` and the
 * trial's fields, frame_pool_bytes), queues n_roots roots whose argument
 * structs lie back to back in root_args (host, args_bytes each, queue 0), runs
 * once to warm up and `reps` more times, and is scored by the median
 * kernel_ms.  Every trial must reproduce the first trial's 16-byte root
 * results exactly, else GTAP_ERR_TASK_FAILED.  trials (host, may be NULL)
 * receives up to max_trials records; *n_trials the number of trials run;
 * *best the chosen configuration.  Device buffers named in the arguments are
 * used by every trial (a program that writes them, e.g. mergesort, must be
 * idempotent: src is read only). */
#define GTAP_TUNE_BLOCKS 1
#define GTAP_TUNE_STEAL 2
#define GTAP_TUNE_QUEUES 4
#define GTAP_TUNE_CAPACITY 8
#define GTAP_TUNE_BACKOFF 16

typedef struct {
    int blocks_per_sm, deque_capacity, n_queues, steal_policy;
    float kernel_ms;   /* median persistent-kernel time of the trial */
    int status;        /* gtap_status of the trial */
    int idle_backoff_ns;
    int pad;
} gtap_tune_trial;

gtap_status gtap_autotune(int mode, const char* program, const void* root_args, size_t args_bytes, int n_roots,
                          int n_queues, size_t frame_pool_bytes, const gtap_config* base, int reps, int tune_mask,
                          gtap_tune_trial* trials, int max_trials, int* n_trials, gtap_tune_trial* best);

/* ------------------------------------------------------------------------
 * Laplace FMM pipeline (Sec. 6.4.1): adaptive octree construction, upward
 * pass, interaction-list construction by dual-tree traversal (DTT) as
 * block-mode tasks of the "fmm_dtt" program, then data-parallel M2L, downward
 * pass and P2P/L2P.  phi_i approximates sum_{j != i} q_j / |x_i - x_j|.
 *
 * Readings fixed by this library (the paper leaves them open): the root cell
 * is the bounding cube of the points; a cell with more than leaf_size points
 * (and level < 21) splits into its non-empty octants, numbered breadth first
 * in Morton order; expansions are Cartesian Taylor series of total order p
 * about cell centres, M2L keeping the terms with |alpha| + |beta| <= p; the
 * MAC accepts a pair (A, B), A != B, iff (R_A + R_B) < theta |c_A - c_B| with
 * R the half-diagonal of the cell cube; a rejected pair of two leaves goes to
 * the P2P list, otherwise the cell of lower level is split (both when the
 * levels are equal).  Lists hold one-directional (target, source) pairs.
 * ---------------------------------------------------------------------- */
#define GTAP_FMM_FP64 0   /* every kernel in FP64 */
#define GTAP_FMM_MIXED 1  /* P2M, M2L, L2P, P2P and the deeper M2M/L2L in FP32, the M2L and
                             P2P sums compensated (Kahan); M2M/L2L into cells of the top
                             fp64_levels levels in FP64.  Expansions are stored in FP64. */

typedef struct {
    int order;             /* expansion order p, 1..8 (default 6) */
    int leaf_size;         /* points per leaf, 1..64 (default 64) */
    double theta;          /* MAC parameter, 0 < theta < 1 (default 0.5) */
    int precision;         /* GTAP_FMM_FP64 (default) or GTAP_FMM_MIXED */
    int fp64_levels;       /* mixed form: translations whose parent is on a level below this
                              number run in FP64 (default 3) */
    int64_t m2l_capacity;  /* list capacities in entries; 0 = from the tree: ceil(128/theta^3)
                              per cell and ceil(32/theta^3) per leaf; an overflow grows the
                              lists (kept for later builds) and repeats the traversal once */
    int64_t p2p_capacity;
    void* stream;          /* cudaStream_t of the data-parallel kernels; use the same stream as
                              the traversal context (default: the legacy default stream) */
} gtap_fmm_config;

typedef struct {
    int64_t n_points, n_cells, n_leaves;
    int n_levels, order;
    int64_t n_m2l, n_p2p;              /* entries produced by the last traversal */
    int64_t m2l_capacity, p2p_capacity;
    float ms_tree, ms_upward;          /* phases of the last build (CUDA events) */
    float ms_traverse;                 /* the traversal's persistent kernel */
    float ms_group, ms_m2l, ms_downward, ms_leaf;   /* phases of the last evaluation */
} gtap_fmm_info;

typedef struct gtap_fmm gtap_fmm;   /* opaque plan: tree, expansions, lists (device) */

/* "fmm_dtt" root argument (block mode): traverse from the cell pair
 * (target, source) of a built plan, appending to the plan's lists. */
typedef struct { const gtap_fmm* plan; int32_t target, source; } gtap_fmm_dtt_args;

/* Create a plan (cfg may be NULL for all defaults).  Builds the expansion
 * tables; device memory is allocated by gtap_fmm_build as sizes become known.
 * Errors: GTAP_ERR_INVALID_ARG, GTAP_ERR_NO_MEMORY. */
gtap_status gtap_fmm_create(const gtap_fmm_config* cfg, gtap_fmm** out);
/* Build the octree and the multipole expansions (octree, P2M, M2M) for n
 * points: pos (device, n x 3 FP64, row-major) and q (device, n FP64), both
 * caller owned and read during the call only.  1 <= n < 2^31; more than 64
 * points sharing one cell of the deepest level (21) is GTAP_ERR_INVALID_ARG.  Grows the
 * plan's device buffers when needed (cudaMalloc); returns after completion.
 * The cell records are checked on the device (bounds, then child links) before
 * any later kernel follows them; a failed check is GTAP_ERR_TASK_FAILED.
 * Errors: GTAP_ERR_INVALID_ARG, GTAP_ERR_NO_MEMORY, GTAP_ERR_CUDA, GTAP_ERR_TASK_FAILED. */
gtap_status gtap_fmm_build(gtap_fmm* f, const double* pos, const double* q, int64_t n);
/* Build the M2L and P2P lists by running "fmm_dtt" from the root pair on ctx,
 * a block-mode context (gtap_init(GTAP_MODE_BLOCK, 1, ...); 128 threads per
 * block and blocks_per_sm = 6, what the traversal kernel's registers allow, is
 * the fastest GB300 setting measured); the context's pending roots are replaced.  On overflow the lists are grown to the sizes
 * the run counted and the traversal is repeated once.  Errors: those of
 * gtap_run/gtap_wait, GTAP_ERR_LIST_OVERFLOW, GTAP_ERR_INVALID_ARG (plan not
 * built, or ctx not in block mode). */
gtap_status gtap_fmm_traverse(gtap_fmm* f, gtap_ctx* ctx);
/* M2L, L2L, L2P and P2P: writes phi (device, n FP64, input point order,
 * caller owned).  Needs a completed traversal.  Returns after completion. */
gtap_status gtap_fmm_evaluate(gtap_fmm* f, double* phi);
/* gtap_fmm_build + gtap_fmm_traverse + gtap_fmm_evaluate. */
gtap_status gtap_fmm_run(gtap_fmm* f, gtap_ctx* ctx, const double* pos, const double* q, int64_t n, double* phi);
gtap_status gtap_fmm_get_info(const gtap_fmm* f, gtap_fmm_info* out);
/* Host copies of the tree: info[n_cells][4] = {first, count, child_first or -1,
 * level << 8 | n_children}, geom[n_cells][4] = {cx, cy, cz, half side} and
 * order[n] (Morton position -> input index).  Any output may be NULL. */
gtap_status gtap_fmm_copy_tree(const gtap_fmm* f, int32_t* info, double* geom, int32_t* order);
/* Host copies of the lists as (target, source) int32 pairs: m2l[n_m2l][2],
 * p2p[n_p2p][2] (either may be NULL).  GTAP_ERR_LIST_OVERFLOW if the last
 * traversal overflowed. */
gtap_status gtap_fmm_copy_lists(const gtap_fmm* f, int32_t* m2l, int32_t* p2p);
gtap_status gtap_fmm_destroy(gtap_fmm* f);

/* ------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart to this call.
 *
 * gtap_mergesort_noalloc sorts n uint32 keys from src into dst (both device
 * pointers owned by the caller; src may equal dst) with the block-mode
 * mergesort above, for callers that cannot allocate device memory: plugins
 * and libraries loaded into a host application that owns all device memory
 * and hands them only a stream and buffers, real-time paths whose memory
 * budget is fixed before they start, and code running under an allocator
 * that must not be re-entered.  All working memory (key scratch, task
 * records, deques, control words) lives in one fixed file-scope device array
 * of about 10 MB, which every GPU that loads the library holds until the
 * process exits; the call makes no cudaMalloc or cudaFree and uses no
 * allocating library routine.
 *   - n must be at most 2^20 (1,048,576); larger n returns GTAP_ERR_INVALID_ARG.
 *   - The first call on a device sets that device up (it looks up the array's
 *     device address); make that first call before any stream capture.
 *   - stream is a cudaStream_t (NULL: the legacy default stream).  The call
 *     returns after the sort has finished on that stream, with the device-side
 *     status (GTAP_ERR_POOL_EXHAUSTED, GTAP_ERR_DEQUE_OVERFLOW, ...) or GTAP_OK.
 *   - All calls share the array, which keeps the previous call's contents;
 *     every run re-initialises what it reads.  Calls whose GPU work overlaps
 *     (different streams or host threads at the same time) race on the array
 *     and are not allowed.
 * ---------------------------------------------------------------------- */
gtap_status gtap_mergesort_noalloc(const uint32_t* src, uint32_t* dst, uint64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GTAP_H_ */
