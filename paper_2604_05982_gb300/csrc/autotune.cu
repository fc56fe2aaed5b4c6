// Autotuner of the launch configuration (batching and tuning, one of the
// systems patterns the runtime takes on): for one program and one batch of
// roots it picks blocks per SM, ring (deque) capacity, DAQ queue count, steal
// policy and the idle back-off by coordinate descent, timing the persistent kernel of each
// trial (median of `reps` runs after one warm-up).  Built on the public calls
// only; every trial must reproduce the root results of the first trial byte
// for byte, so a configuration can change speed but never an answer.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gtap.h"

namespace {

struct Trial {
    int bps, cap, queues, steal, backoff;
};

struct Tuner {
    int mode;
    const char* program;
    const unsigned char* args;
    size_t args_bytes;
    int n_roots;
    size_t pool_bytes;
    gtap_config base;
    int reps;
    std::vector<unsigned char> ref;   // root results of the first successful trial
    bool have_ref = false;
    gtap_tune_trial* out;
    int max_out, n_out = 0;

    gtap_status run(const Trial& tr, float* ms) {
        gtap_config cfg = base;
        cfg.blocks_per_sm = tr.bps;
        cfg.deque_capacity = tr.cap;
        cfg.steal_policy = tr.steal;
        cfg.idle_backoff_ns = tr.backoff;
        gtap_ctx* c = nullptr;
        gtap_status st = gtap_init((gtap_mode)mode, tr.queues, pool_bytes, &cfg, &c);
        if (st != GTAP_OK) return st;
        int type = 0;
        std::vector<uint64_t> handles((size_t)n_roots);
        st = gtap_register_task(c, program, &type);
        for (int r = 0; st == GTAP_OK && r < n_roots; ++r)
            st = gtap_spawn_root(c, type, args + (size_t)r * args_bytes, args_bytes, 0, &handles[(size_t)r]);
        std::vector<float> times;
        for (int it = 0; st == GTAP_OK && it <= reps; ++it) {
            st = gtap_run(c);
            if (st == GTAP_OK) st = gtap_wait(c, 0);
            gtap_stats s;
            if (st == GTAP_OK && it > 0 && gtap_get_stats(c, &s) == GTAP_OK) times.push_back(s.kernel_ms);
        }
        if (st == GTAP_OK) {
            std::vector<unsigned char> res((size_t)n_roots * 16);
            for (int r = 0; st == GTAP_OK && r < n_roots; ++r)
                st = gtap_read_result(c, handles[(size_t)r], res.data() + (size_t)r * 16, 16);
            if (st == GTAP_OK) {
                if (!have_ref) {
                    ref = res;
                    have_ref = true;
                } else if (res != ref) {
                    st = GTAP_ERR_TASK_FAILED;   // a configuration changed an answer
                }
            }
        }
        gtap_finalize(c);
        std::sort(times.begin(), times.end());
        *ms = times.empty() ? 0.f : times[times.size() / 2];
        if (n_out < max_out && out) {
            gtap_tune_trial& t = out[n_out];
            t.blocks_per_sm = tr.bps;
            t.deque_capacity = tr.cap;
            t.n_queues = tr.queues;
            t.steal_policy = tr.steal;
            t.kernel_ms = *ms;
            t.status = (int)st;
            t.idle_backoff_ns = tr.backoff;
            t.pad = 0;
        }
        ++n_out;
        return st;
    }
};

}  // namespace

extern "C" gtap_status gtap_autotune(int mode, const char* program, const void* root_args, size_t args_bytes,
                                     int n_roots, int n_queues, size_t frame_pool_bytes, const gtap_config* base,
                                     int reps, int tune_mask, gtap_tune_trial* trials, int max_trials, int* n_trials,
                                     gtap_tune_trial* best) {
    if ((mode != GTAP_MODE_THREAD && mode != GTAP_MODE_BLOCK) || !program || !root_args || args_bytes == 0 ||
        n_roots < 1 || reps < 1 || !best || max_trials < 0 || n_queues < 1 || n_queues > 8 ||
        (mode == GTAP_MODE_BLOCK && n_queues != 1) || (tune_mask & ~31) != 0)
        return GTAP_ERR_INVALID_ARG;
    if (tune_mask == 0)
        tune_mask = GTAP_TUNE_BLOCKS | GTAP_TUNE_STEAL | GTAP_TUNE_QUEUES | GTAP_TUNE_CAPACITY | GTAP_TUNE_BACKOFF;
    Tuner t;
    t.mode = mode;
    t.program = program;
    t.args = static_cast<const unsigned char*>(root_args);
    t.args_bytes = args_bytes;
    t.n_roots = n_roots;
    t.pool_bytes = frame_pool_bytes;
    std::memset(&t.base, 0, sizeof(t.base));
    if (base) t.base = *base;
    t.reps = reps;
    t.out = trials;
    t.max_out = max_trials;

    const bool thread = mode == GTAP_MODE_THREAD;
    const std::vector<int> bps = thread ? std::vector<int>{1, 2, 4, 6, 8} : std::vector<int>{1, 2, 3, 4, 6};
    const std::vector<int> steal = thread ? std::vector<int>{GTAP_STEAL_FILL, GTAP_STEAL_EMPTY, GTAP_STEAL_HALF,
                                                             GTAP_STEAL_EMPTY | GTAP_STEAL_HALF}
                                          : std::vector<int>{0, GTAP_STEAL_ONE};
    const std::vector<int> queues = thread ? std::vector<int>{1, 2, 3, 4} : std::vector<int>{1};
    const std::vector<int> caps = {1024, 4096, 16384};
    // the idle back-off exists in thread mode only
    const std::vector<int> backoffs = thread ? std::vector<int>{512, 2048, 8192} : std::vector<int>{};

    Trial cur{4, 4096, n_queues, thread ? GTAP_STEAL_FILL : 0, t.base.idle_backoff_ns ? t.base.idle_backoff_ns : 512};
    float cur_ms = 0.f;
    gtap_status st = t.run(cur, &cur_ms);
    if (st != GTAP_OK) {
        if (n_trials) *n_trials = t.n_out;
        return st;
    }
    // coordinate descent, one sweep per parameter in this order
    for (int dim = 0; dim < 5; ++dim) {
        if ((tune_mask & (1 << dim)) == 0) continue;
        const std::vector<int>& vals = dim == 0 ? bps : dim == 1 ? steal : dim == 2 ? queues : dim == 3 ? caps : backoffs;
        const int start = dim == 0 ? cur.bps : dim == 1 ? cur.steal : dim == 2 ? cur.queues : dim == 3 ? cur.cap
                                                                                                      : cur.backoff;
        for (int v : vals) {
            if (v == start) continue;   // already timed
            Trial tr = cur;
            int& field = dim == 0 ? tr.bps : dim == 1 ? tr.steal : dim == 2 ? tr.queues : dim == 3 ? tr.cap : tr.backoff;
            field = v;
            float ms = 0.f;
            gtap_status s = t.run(tr, &ms);
            if (s == GTAP_ERR_TASK_FAILED && t.have_ref) {   // a changed answer is a hard error
                if (n_trials) *n_trials = t.n_out;
                return s;
            }
            if (s == GTAP_OK && ms > 0.f && ms < cur_ms) {
                cur = tr;
                cur_ms = ms;
            }
        }
    }
    best->blocks_per_sm = cur.bps;
    best->deque_capacity = cur.cap;
    best->n_queues = cur.queues;
    best->steal_policy = cur.steal;
    best->idle_backoff_ns = cur.backoff;
    best->pad = 0;
    best->kernel_ms = cur_ms;
    best->status = GTAP_OK;
    if (n_trials) *n_trials = t.n_out;
    return GTAP_OK;
}
