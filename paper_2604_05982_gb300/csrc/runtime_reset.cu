// Per-run reset: re-zero the deques and control words, re-arm the pool's
// chunk queue, write the root records and push each root to a worker's deque
// (Sec. 4: storage is preallocated; a run only re-initialises it).
#include "launch.h"
#include "gtap_device.cuh"

namespace gtap {

__global__ void reset_kernel(KParams P, int init_cq) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    const uint32_t Q = P.n_queues;
    const uint32_t cap = P.ring_mask + 1;
    if (init_cq)
        for (size_t i = tid; i <= P.ncq_mask; i += nth) P.cq_seq[i] = i;
    if (P.sq_seq != nullptr)
        for (size_t i = tid; i <= P.sq_mask; i += nth) P.sq_seq[i] = i;
    if (P.lq_seq != nullptr)
        for (size_t i = tid; i <= P.lq_mask; i += nth) P.lq_seq[i] = i;
    if (P.gq != nullptr) {
        // central queue: slot i holds root i (published: sequence i + 1), the rest are free (sequence i)
        for (size_t i = tid; i <= P.gq_mask; i += nth) {
            const bool root = i < P.n_roots;
            P.gq[i] = ((unsigned long long)(uint32_t)(i + (root ? 1 : 0)) << 32) | (root ? (uint32_t)i : 0u);
        }
    }
    if (P.fstate != nullptr)
        for (size_t i = tid; i < P.n_frames; i += nth) P.fstate[i] = (i < P.n_roots) ? 3u : 0u;
    // root records
    for (size_t r = tid; r < P.n_roots; r += nth) {
        const RootDesc& d = P.root_desc[r];
        char* f = frame_ptr(P, (uint32_t)r);
        FrameHdr h;
        h.w0 = d.type & 0xFFu;
        h.pending = 0;
        h.parent = kRootBit | (uint32_t)r;
        h.w3 = 0;
        *reinterpret_cast<FrameHdr*>(f) = h;
        for (int i = 0; i < kRootPayloadBytes / 4; ++i)
            reinterpret_cast<uint32_t*>(f + kHdrBytes)[i] = reinterpret_cast<const uint32_t*>(d.payload)[i];
        RootEntry e;
        e.result[0] = 0; e.result[1] = 0; e.done = 0; e.type = d.type; e.req = r;
        P.roots[r] = e;
    }
    // deques: worker w owns roots w, w + W, w + 2W, ...
    for (size_t w = tid; w < P.n_workers; w += nth) {
        uint32_t cnt[kMaxQueues];
        for (uint32_t q = 0; q < Q; ++q) cnt[q] = 0;
        for (size_t r = w; P.gq == nullptr && r < P.n_roots; r += P.n_workers) {
            const uint32_t q = P.root_desc[r].queue % Q;
            P.rings[((size_t)w * Q + q) * cap + cnt[q]] = (uint32_t)r;
            ++cnt[q];
        }
        for (uint32_t q = 0; q < Q; ++q) {
            QState s;
            s.count = (int)cnt[q];
            s.head = 0;
            s.lock = 0;
            s.tail0 = cnt[q];
            P.qs[(size_t)w * Q + q] = s;
        }
    }
    if (tid == 0) {
        P.ctl->roots_remaining.v = P.n_roots;
        P.ctl->abort_flag.v = 0;
        P.ctl->bump.v = P.n_roots;
        P.ctl->cq_enq.v = 0;
        P.ctl->cq_deq.v = 0;
        P.ctl->cq_avail.v = 0;
        P.ctl->sc_enq.v = 0;
        P.ctl->sc_deq.v = 0;
        P.ctl->sc_avail.v = 0;
        P.ctl->lc_enq.v = 0;
        P.ctl->lc_deq.v = 0;
        P.ctl->lc_avail.v = 0;
        P.ctl->out_tail.v = 0;
        P.ctl->admitted.v = 0;
        P.ctl->scratch_top.v = 0;
        P.ctl->inflight.v = 0;
        P.ctl->gq_enq.v = P.gq ? P.n_roots : 0;
        P.ctl->gq_deq.v = 0;
        P.ctl->gq_avail.v = P.gq ? P.n_roots : 0;
        P.ctl->err.code = 0;
        P.ctl->err.task_type = -1;
        P.ctl->err.worker = -1;
        P.ctl->err.detail = 0;
    }
}

cudaError_t launch_reset(const KParams& P, int init_cq, cudaStream_t s) {
    reset_kernel<<<304, 256, 0, s>>>(P, init_cq);
    return cudaGetLastError();
}

}  // namespace gtap
