// Host side of the Laplace FMM pipeline (Sec. 6.4.1) behind the C ABI: the
// plan object, the expansion tables, buffer management and the phase order
// tree -> upward pass -> traversal (fmm_dtt tasks) -> M2L -> downward pass ->
// leaf kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "fmm_internal.h"
#include "gtap.h"
#include "scan.cuh"

using namespace gtap;
using namespace gtap::fmm;

namespace {

struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    bool ensure(size_t want) {
        if (want <= bytes && p) return true;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (cudaMalloc(&p, std::max<size_t>(want, 256)) != cudaSuccess) { p = nullptr; return false; }
        bytes = std::max<size_t>(want, 256);
        return true;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

struct HostTables {
    int p = 0, nt = 0;
    std::vector<short3> mi;
    std::vector<DerivEntry> deriv;
    std::vector<ItemEntry> items;
    std::vector<int> item_off;
    std::vector<TermEntry> m2l, m2m, l2l;
    std::vector<int> m2m_off, l2l_off;
    std::vector<double> mscale, lscale;   // (-1)^|a| / a!  and  1 / b!  per coefficient

    int at(int a, int b, int c) const {
        if (a < 0 || b < 0 || c < 0 || a + b + c > p) return -1;
        for (int i = 0; i < nt; ++i)
            if (mi[i].x == a && mi[i].y == b && mi[i].z == c) return i;
        return -1;
    }
    static TermEntry term(int a, int b, double coef) {
        TermEntry t;
        t.a = (uint8_t)a;
        t.b = (uint8_t)b;
        t.pad = 0;
        t.coef32 = (float)coef;
        t.coef64 = coef;
        return t;
    }
    void build(int order) {
        p = order;
        for (int k = 0; k <= p; ++k)
            for (int a = k; a >= 0; --a)
                for (int b = k - a; b >= 0; --b) mi.push_back(make_short3((short)a, (short)b, (short)(k - a - b)));
        nt = (int)mi.size();
        for (int i = 0; i < nt; ++i) {
            const int a = mi[i].x, b = mi[i].y, c = mi[i].z;
            DerivEntry d;
            d.e1[0] = (short)at(a - 1, b, c); d.e1[1] = (short)at(a, b - 1, c); d.e1[2] = (short)at(a, b, c - 1);
            d.e2[0] = (short)at(a - 2, b, c); d.e2[1] = (short)at(a, b - 2, c); d.e2[2] = (short)at(a, b, c - 2);
            d.k = (short)(a + b + c);
            d.pad = 0;
            deriv.push_back(d);
            double fa = 1.0;
            for (int t = 2; t <= a; ++t) fa *= t;
            for (int t = 2; t <= b; ++t) fa *= t;
            for (int t = 2; t <= c; ++t) fa *= t;
            lscale.push_back(1.0 / fa);
            mscale.push_back(((a + b + c) & 1) ? -1.0 / fa : 1.0 / fa);
        }
        // M2L: for each beta, the alphas with |alpha| + |beta| <= p, in chunks
        for (int bi = 0; bi < nt; ++bi) {
            const short3 be = mi[bi];
            item_off.push_back((int)items.size());
            const int first = (int)m2l.size();
            for (int ai = 0; ai < nt; ++ai) {
                const short3 al = mi[ai];
                if (al.x + al.y + al.z + be.x + be.y + be.z > p) continue;
                const double sign = ((al.x + al.y + al.z) & 1) ? -1.0 : 1.0;
                const double cab = binom(al.x + be.x, be.x) * binom(al.y + be.y, be.y) * binom(al.z + be.z, be.z);
                m2l.push_back(term(ai, at(al.x + be.x, al.y + be.y, al.z + be.z), sign * cab));
            }
            const int last = (int)m2l.size();
            for (int s = first; s < last; s += kM2lChunk) {
                ItemEntry it;
                it.out = (uint16_t)bi;
                it.first = (uint16_t)s;
                it.len = (uint16_t)std::min(kM2lChunk, last - s);
                it.pad = 0;
                items.push_back(it);
            }
        }
        item_off.push_back((int)items.size());
        // M2M: for each alpha, beta <= alpha; L2L: for each gamma, beta >= gamma
        for (int ai = 0; ai < nt; ++ai) {
            const short3 al = mi[ai];
            m2m_off.push_back((int)m2m.size());
            l2l_off.push_back((int)l2l.size());
            for (int bi = 0; bi < nt; ++bi) {
                const short3 be = mi[bi];
                if (be.x <= al.x && be.y <= al.y && be.z <= al.z)
                    m2m.push_back(term(bi, at(al.x - be.x, al.y - be.y, al.z - be.z),
                                       binom(al.x, be.x) * binom(al.y, be.y) * binom(al.z, be.z)));
                if (be.x >= al.x && be.y >= al.y && be.z >= al.z)
                    l2l.push_back(term(bi, at(be.x - al.x, be.y - al.y, be.z - al.z),
                                       binom(be.x, al.x) * binom(be.y, al.y) * binom(be.z, al.z)));
            }
        }
        m2m_off.push_back((int)m2m.size());
        l2l_off.push_back((int)l2l.size());
    }
};

template <class T>
size_t put(std::vector<unsigned char>& blob, const std::vector<T>& v) {
    size_t off = (blob.size() + 15) & ~size_t(15);
    blob.resize(off + v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

}  // namespace

struct gtap_fmm {
    gtap_fmm_config cfg{};
    int p = 6, nt = 84;
    bool mixed = false;
    cudaStream_t s = nullptr;
    HostTables ht;
    Tables tab{};
    DBuf tab_dev;

    // tree
    DBuf keys0, keys1, vals0, vals1, pts, ploc, hist, hist_scan, tile_sums, box, bbox_part, geom, info, lat, lstart,
        lvl_n, lvl_total, cnt, off, bounds, flags;
    double box_h[8] = {};
    int cell_cap = 0;
    const uint32_t* order = nullptr;
    // expansions and lists
    DBuf M, L, m2l, p2p, counters, gcnt, gcur, m2l_off, m2l_src, p2p_off, p2p_src, ms, aux;
    long long m2l_cap = 0, p2p_cap = 0;

    long long n = 0;
    int n_cells = 0, n_leaves = 0, n_levels = 0;
    int lstart_h[kMaxLevel + 3] = {};
    bool built = false, traversed = false;
    long long n_m2l = 0, n_p2p = 0;
    gtap_fmm_info info_h{};
    cudaEvent_t ev[8] = {};

    ~gtap_fmm() {
        DBuf* all[] = {&tab_dev, &keys0, &keys1, &vals0, &vals1, &pts, &ploc, &hist, &hist_scan, &tile_sums, &box,
                       &bbox_part, &geom, &info, &lat, &lstart, &lvl_n, &lvl_total, &cnt, &off, &bounds, &flags, &M, &L,
                       &m2l, &p2p, &counters, &gcnt, &gcur, &m2l_off, &m2l_src, &p2p_off, &p2p_src, &ms, &aux};
        for (DBuf* b : all) b->release();
        for (cudaEvent_t& e : ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? ms : 0.f;
}

// Make the lists hold at least the given entries.  A capacity never drops below
// what is already allocated, so a size learned from an overflow is kept for
// later builds of the plan.
gtap_status grow_lists(gtap_fmm* f, long long m2l_cap, long long p2p_cap) {
    const long long lim = (1ll << 31) - 1;
    m2l_cap = std::min(std::max(m2l_cap, 1ll), lim);
    p2p_cap = std::min(std::max(p2p_cap, 1ll), lim);
    if (!f->m2l.ensure(sizeof(unsigned long long) * (size_t)m2l_cap) ||
        !f->p2p.ensure(sizeof(unsigned long long) * (size_t)p2p_cap))
        return GTAP_ERR_NO_MEMORY;
    f->m2l_cap = std::min(lim, (long long)(f->m2l.bytes / sizeof(unsigned long long)));
    f->p2p_cap = std::min(lim, (long long)(f->p2p.bytes / sizeof(unsigned long long)));
    return GTAP_OK;
}

EvalBufs eval_bufs(gtap_fmm* f, double* phi) {
    EvalBufs e;
    e.p = f->p;
    e.nt = f->nt;
    e.n_cells = f->n_cells;
    e.n_levels = f->n_levels;
    e.n = f->n;
    e.geom = f->geom.as<Dbl4>();
    e.info = f->info.as<int4>();
    e.lat = f->lat.as<int4>();
    e.lat_unit = (float)(f->box_h[3] / 4194304.0);
    e.lstart = f->lstart_h;
    e.pts = f->pts.as<Dbl4>();
    e.ploc = f->ploc.as<float4>();
    e.order = f->order;
    e.M = f->M.as<double>();
    e.L = f->L.as<double>();
    e.tab = f->tab;
    e.m2l_off = f->m2l_off.as<int>();
    e.m2l_src = f->m2l_src.as<int>();
    e.p2p_off = f->p2p_off.as<int>();
    e.p2p_src = f->p2p_src.as<int>();
    e.phi = phi;
    e.m2l_ms = f->ms.p;
    return e;
}

}  // namespace

namespace gtap {
namespace fmm {

gtap_status dtt_env(const gtap_fmm* f, int target, int source, DttEnv* out) {
    if (!f || !out || !f->built) return GTAP_ERR_INVALID_ARG;
    if (target < 0 || source < 0 || target >= f->n_cells || source >= f->n_cells) return GTAP_ERR_INVALID_ARG;
    out->geom = f->geom.as<Dbl4>();
    out->info = f->info.as<int4>();
    out->lat = f->lat.as<int4>();
    out->m2l = f->m2l.as<unsigned long long>();
    out->p2p = f->p2p.as<unsigned long long>();
    out->counters = f->counters.as<unsigned long long>();
    out->aux = f->aux.as<DttAux>();
    out->n_cells = f->n_cells;
    out->pad = 0;
    return GTAP_OK;
}

}  // namespace fmm
}  // namespace gtap

extern "C" {

gtap_status gtap_fmm_create(const gtap_fmm_config* cfg, gtap_fmm** out) {
    if (!out) return GTAP_ERR_INVALID_ARG;
    *out = nullptr;
    gtap_fmm_config c{};
    if (cfg) c = *cfg;
    if (c.order == 0) c.order = 6;
    if (c.leaf_size == 0) c.leaf_size = 64;
    if (c.theta == 0.0) c.theta = 0.5;
    if (c.fp64_levels == 0) c.fp64_levels = 3;
    if (c.order < 1 || c.order > kMaxOrder || c.leaf_size < 1 || c.leaf_size > kMaxLeaf || !(c.theta > 0.0) ||
        !(c.theta < 1.0) || (c.precision != GTAP_FMM_FP64 && c.precision != GTAP_FMM_MIXED) || c.fp64_levels < 0 ||
        c.m2l_capacity < 0 || c.p2p_capacity < 0)
        return GTAP_ERR_INVALID_ARG;
    gtap_fmm* f = new (std::nothrow) gtap_fmm;
    if (!f) return GTAP_ERR_NO_MEMORY;
    f->cfg = c;
    f->p = c.order;
    f->mixed = c.precision == GTAP_FMM_MIXED;
    f->s = static_cast<cudaStream_t>(c.stream);
    f->ht.build(c.order);
    f->nt = f->ht.nt;
    const HostTables& h = f->ht;
    std::vector<unsigned char> blob;
    const size_t o_mi = put(blob, h.mi), o_der = put(blob, h.deriv), o_items = put(blob, h.items),
                 o_ioff = put(blob, h.item_off), o_m2l = put(blob, h.m2l), o_m2mo = put(blob, h.m2m_off),
                 o_m2m = put(blob, h.m2m), o_l2lo = put(blob, h.l2l_off), o_l2l = put(blob, h.l2l),
                 o_ms = put(blob, h.mscale), o_ls = put(blob, h.lscale);
    if (!f->tab_dev.ensure(blob.size()) ||
        cudaMemcpy(f->tab_dev.p, blob.data(), blob.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        delete f;
        return GTAP_ERR_NO_MEMORY;
    }
    unsigned char* base = f->tab_dev.as<unsigned char>();
    Tables& t = f->tab;
    t.p = f->p;
    t.nt = f->nt;
    t.n_m2l_items = (int)h.items.size();
    t.n_m2l_terms = (int)h.m2l.size();
    t.n_shift_terms = (int)h.m2m.size();
    t.mi = reinterpret_cast<short3*>(base + o_mi);
    t.deriv = reinterpret_cast<DerivEntry*>(base + o_der);
    t.m2l_items = reinterpret_cast<ItemEntry*>(base + o_items);
    t.m2l_item_off = reinterpret_cast<int*>(base + o_ioff);
    t.m2l_terms = reinterpret_cast<TermEntry*>(base + o_m2l);
    t.m2m_off = reinterpret_cast<int*>(base + o_m2mo);
    t.m2m_terms = reinterpret_cast<TermEntry*>(base + o_m2m);
    t.l2l_off = reinterpret_cast<int*>(base + o_l2lo);
    t.l2l_terms = reinterpret_cast<TermEntry*>(base + o_l2l);
    t.mscale = reinterpret_cast<double*>(base + o_ms);
    t.lscale = reinterpret_cast<double*>(base + o_ls);
    for (cudaEvent_t& e : f->ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            delete f;
            return GTAP_ERR_CUDA;
        }
    if (!f->counters.ensure(4 * sizeof(unsigned long long)) || !f->aux.ensure(sizeof(DttAux)) ||
        !f->box.ensure(8 * sizeof(double)) ||
        !f->bbox_part.ensure(6 * kBoxParts * sizeof(double)) || !f->lstart.ensure((kMaxLevel + 3) * sizeof(int)) ||
        !f->lvl_n.ensure((kMaxLevel + 1) * sizeof(int)) || !f->lvl_total.ensure((kMaxLevel + 1) * sizeof(int)) ||
        !f->flags.ensure(4 * sizeof(int))) {
        delete f;
        return GTAP_ERR_NO_MEMORY;
    }
    *out = f;
    return GTAP_OK;
}

gtap_status gtap_fmm_build(gtap_fmm* f, const double* pos, const double* q, int64_t n) {
    if (!f || !pos || !q || n < 1 || n >= (1ll << 31) - 1) return GTAP_ERR_INVALID_ARG;
    f->built = f->traversed = false;
    const size_t N = (size_t)n;
    const int ntiles = radix_tiles(n);
    if (!f->keys0.ensure(8 * N) || !f->keys1.ensure(8 * N) || !f->vals0.ensure(4 * N) || !f->vals1.ensure(4 * N) ||
        !f->pts.ensure(sizeof(Dbl4) * N) || !f->hist.ensure(sizeof(int) * 256 * (size_t)ntiles) ||
        !f->hist_scan.ensure(sizeof(int) * 256 * (size_t)ntiles) || (f->mixed && !f->ploc.ensure(sizeof(float4) * N)))
        return GTAP_ERR_NO_MEMORY;
    // cell capacity: a first guess, doubled while a level does not fit
    long long cap = std::max<long long>(1024, 2 * (8 * n / (f->cfg.leaf_size + 1)) + 64);
    cap = std::max<long long>(cap, f->cell_cap);
    cudaEventRecord(f->ev[0], f->s);
    for (int attempt = 0;; ++attempt) {
        if (cap >= (1ll << 31) / 9) return GTAP_ERR_NO_MEMORY;
        const size_t C = (size_t)cap;
        if (!f->geom.ensure(sizeof(Dbl4) * C) || !f->info.ensure(sizeof(int4) * C) || !f->lat.ensure(sizeof(int4) * C) ||
            !f->cnt.ensure(sizeof(int) * C) ||
            !f->off.ensure(sizeof(int) * C) || !f->bounds.ensure(sizeof(int) * 9 * C) ||
            !f->tile_sums.ensure(sizeof(int) * (size_t)scan::tiles_for(std::max<long long>(cap, 256ll * ntiles))))
            return GTAP_ERR_NO_MEMORY;
        f->cell_cap = (int)cap;
        TreeBufs b{};
        b.n = n;
        b.leaf = f->cfg.leaf_size;
        b.pos = pos;
        b.q = q;
        b.box = f->box.as<double>();
        b.bbox_part = f->bbox_part.as<double>();
        b.keys[0] = f->keys0.as<unsigned long long>();
        b.keys[1] = f->keys1.as<unsigned long long>();
        b.vals[0] = f->vals0.as<uint32_t>();
        b.vals[1] = f->vals1.as<uint32_t>();
        b.hist = f->hist.as<int>();
        b.hist_scan = f->hist_scan.as<int>();
        b.tile_sums = f->tile_sums.as<int>();
        b.geom = f->geom.as<Dbl4>();
        b.info = f->info.as<int4>();
        b.lat = f->lat.as<int4>();
        b.cap_cells = (int)cap;
        b.lstart = f->lstart.as<int>();
        b.lvl_n = f->lvl_n.as<int>();
        b.lvl_total = f->lvl_total.as<int>();
        b.cnt = f->cnt.as<int>();
        b.off = f->off.as<int>();
        b.bounds = f->bounds.as<int>();
        b.flags = f->flags.as<int>();
        b.pts = f->pts.as<Dbl4>();
        b.ploc = f->ploc.as<float4>();
        if (launch_tree_sort(b, f->s) != cudaSuccess) return GTAP_ERR_CUDA;
        // Refine level by level.  A level without cells ends the tree, so between
        // chunks of levels the host looks at the next level's size and stops at the
        // first empty one (a uniform 2^20 set has 6 levels, a Plummer set 10, of 21).
        int done = 0;
        for (int chunk : {8, 4, 4, 5}) {
            const int l1 = std::min(done + chunk, kMaxLevel);
            if (launch_tree_levels(b, done, l1, f->s) != cudaSuccess) return GTAP_ERR_CUDA;
            done = l1;
            if (done >= kMaxLevel) break;
            int ls[2] = {0, 0};   // the cells of level `done`: [ls[0], ls[1])
            if (cudaMemcpyAsync(ls, f->lstart.as<int>() + done, sizeof(ls), cudaMemcpyDeviceToHost, f->s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(f->s) != cudaSuccess)
                return GTAP_ERR_CUDA;
            if (ls[1] == ls[0]) break;
        }
        if (launch_tree_finish(b, done, f->s) != cudaSuccess) return GTAP_ERR_CUDA;
        int flags[4] = {0, 0, 0, 0};
        if (cudaMemcpyAsync(flags, f->flags.p, sizeof(flags), cudaMemcpyDeviceToHost, f->s) != cudaSuccess ||
            cudaMemcpyAsync(f->lstart_h, f->lstart.p, sizeof(f->lstart_h), cudaMemcpyDeviceToHost, f->s) != cudaSuccess ||
            cudaMemcpyAsync(f->box_h, f->box.p, sizeof(f->box_h), cudaMemcpyDeviceToHost, f->s) != cudaSuccess ||
            cudaStreamSynchronize(f->s) != cudaSuccess)
            return GTAP_ERR_CUDA;
        f->order = b.order;
        if (!flags[0]) {
            // the records were checked on the device before any later kernel follows their links
            if (flags[1]) return GTAP_ERR_TASK_FAILED;
            // only a cell of the deepest level can exceed leaf_size: more than
            // kMaxLeaf points sharing one 21-bit Morton code are not supported
            if (flags[3] > kMaxLeaf) return GTAP_ERR_INVALID_ARG;
            f->n_cells = f->lstart_h[kMaxLevel + 1];
            f->n_leaves = flags[2];
            if (f->mixed && launch_leaf_local(b, f->n_cells, f->s) != cudaSuccess) return GTAP_ERR_CUDA;
            break;
        }
        cap *= 2;
    }
    f->n = n;
    f->n_levels = 0;
    for (int l = 0; l <= kMaxLevel; ++l)
        if (f->lstart_h[l + 1] > f->lstart_h[l]) f->n_levels = l + 1;
    cudaEventRecord(f->ev[1], f->s);
    const size_t ncoef = (size_t)f->n_cells * f->nt;
    if (!f->M.ensure(sizeof(double) * ncoef) || !f->L.ensure(sizeof(double) * ncoef)) return GTAP_ERR_NO_MEMORY;
    EvalBufs e = eval_bufs(f, nullptr);
    if (launch_upward(e, f->mixed, f->cfg.fp64_levels, f->s) != cudaSuccess) return GTAP_ERR_CUDA;
    cudaEventRecord(f->ev[2], f->s);
    // list capacities
    const double th3 = f->cfg.theta * f->cfg.theta * f->cfg.theta;
    long long mc = f->cfg.m2l_capacity ? f->cfg.m2l_capacity : (long long)f->n_cells * (long long)std::ceil(128.0 / th3);
    long long pc = f->cfg.p2p_capacity ? f->cfg.p2p_capacity : (long long)f->n_leaves * (long long)std::ceil(32.0 / th3);
    gtap_status st = grow_lists(f, mc, pc);
    if (st != GTAP_OK) return st;
    if (cudaStreamSynchronize(f->s) != cudaSuccess) return GTAP_ERR_CUDA;
    f->built = true;
    f->info_h.ms_tree = elapsed(f->ev[0], f->ev[1]);
    f->info_h.ms_upward = elapsed(f->ev[1], f->ev[2]);
    return GTAP_OK;
}

gtap_status gtap_fmm_traverse(gtap_fmm* f, gtap_ctx* ctx) {
    if (!f || !ctx || !f->built) return GTAP_ERR_INVALID_ARG;
    f->traversed = false;
    int type = 0;
    gtap_status st = gtap_register_task(ctx, "fmm_dtt", &type);
    if (st != GTAP_OK) return st;
    for (int attempt = 0; attempt < 2; ++attempt) {
        // traversal constants: theta, capacities, and whether the FP32 screen of the MAC is safe.
        // Centres carry FP64 rounding of about 2^-52 |c|; a nonzero centre difference is at least
        // side / 2^21, so the relative gap to the exact lattice values is at most ~2^-50 (|c|max /
        // side) 2^21, which must stay far below the 1e-5 screening margin.
        DttAux ax{};
        ax.theta = f->cfg.theta;
        ax.theta2 = (float)(f->cfg.theta * f->cfg.theta);
        ax.margin = 1e-5f;
        ax.m2l_cap = f->m2l_cap;
        ax.p2p_cap = f->p2p_cap;
        double cmax = 0.0;
        for (int d = 0; d < 3; ++d) cmax = std::max(cmax, std::max(std::fabs(f->box_h[d]), std::fabs(f->box_h[d] + f->box_h[3])));
        const double gap = std::ldexp(1.0, -50) * (cmax / f->box_h[3]) * std::ldexp(1.0, 21);
        ax.screen = gap < 1e-6 ? 1 : 0;
        if (cudaMemcpyAsync(f->aux.p, &ax, sizeof(ax), cudaMemcpyHostToDevice, f->s) != cudaSuccess ||
            cudaMemsetAsync(f->counters.p, 0, 4 * sizeof(unsigned long long), f->s) != cudaSuccess ||
            cudaStreamSynchronize(f->s) != cudaSuccess)
            return GTAP_ERR_CUDA;
        if ((st = gtap_clear_roots(ctx)) != GTAP_OK) return st;
        gtap_fmm_dtt_args a{f, 0, 0};
        if ((st = gtap_spawn_root(ctx, type, &a, sizeof(a), 0, nullptr)) != GTAP_OK) return st;
        if ((st = gtap_run(ctx)) != GTAP_OK) return st;
        if ((st = gtap_wait(ctx, 0)) != GTAP_OK) return st;
        gtap_stats stats;
        if (gtap_get_stats(ctx, &stats) == GTAP_OK) f->info_h.ms_traverse = stats.kernel_ms;
        unsigned long long cnt[2] = {0, 0};
        if (cudaMemcpy(cnt, f->counters.p, sizeof(cnt), cudaMemcpyDeviceToHost) != cudaSuccess) return GTAP_ERR_CUDA;
        f->n_m2l = (long long)cnt[0];
        f->n_p2p = (long long)cnt[1];
        if (f->n_m2l <= f->m2l_cap && f->n_p2p <= f->p2p_cap) {
            f->traversed = true;
            return GTAP_OK;
        }
        if (attempt == 0) {
            st = grow_lists(f, std::max(f->m2l_cap, f->n_m2l + f->n_m2l / 8), std::max(f->p2p_cap, f->n_p2p + f->n_p2p / 8));
            if (st != GTAP_OK) return st;
        }
    }
    return GTAP_ERR_LIST_OVERFLOW;
}

gtap_status gtap_fmm_evaluate(gtap_fmm* f, double* phi) {
    if (!f || !phi || !f->built || !f->traversed) return GTAP_ERR_INVALID_ARG;
    const size_t nc = (size_t)f->n_cells;
    if (!f->gcnt.ensure(sizeof(int) * nc) || !f->gcur.ensure(sizeof(int) * nc) ||
        !f->m2l_off.ensure(sizeof(int) * (nc + 1)) || !f->p2p_off.ensure(sizeof(int) * (nc + 1)) ||
        !f->m2l_src.ensure(sizeof(int) * (size_t)std::max(f->n_m2l, 1ll)) ||
        !f->p2p_src.ensure(sizeof(int) * (size_t)std::max(f->n_p2p, 1ll)) ||
        !f->tile_sums.ensure(sizeof(int) * (size_t)scan::tiles_for((long long)nc)) ||
        !f->ms.ensure(m2l_scratch_bytes(f->p, f->n_cells, f->mixed)))
        return GTAP_ERR_NO_MEMORY;
    cudaEventRecord(f->ev[3], f->s);
    if (launch_group(f->m2l.as<unsigned long long>(), f->n_m2l, f->n_cells, f->gcnt.as<int>(), f->m2l_off.as<int>(),
                     f->gcur.as<int>(), f->m2l_src.as<int>(), f->tile_sums.as<int>(), f->s) != cudaSuccess ||
        launch_group(f->p2p.as<unsigned long long>(), f->n_p2p, f->n_cells, f->gcnt.as<int>(), f->p2p_off.as<int>(),
                     f->gcur.as<int>(), f->p2p_src.as<int>(), f->tile_sums.as<int>(), f->s) != cudaSuccess)
        return GTAP_ERR_CUDA;
    cudaEventRecord(f->ev[4], f->s);
    if (cudaMemsetAsync(f->L.p, 0, sizeof(double) * nc * f->nt, f->s) != cudaSuccess) return GTAP_ERR_CUDA;
    EvalBufs e = eval_bufs(f, phi);
    if (launch_m2l(e, f->mixed, f->s) != cudaSuccess) return GTAP_ERR_CUDA;
    cudaEventRecord(f->ev[5], f->s);
    if (launch_downward(e, f->mixed, f->cfg.fp64_levels, f->s) != cudaSuccess) return GTAP_ERR_CUDA;
    cudaEventRecord(f->ev[6], f->s);
    if (launch_leaf_eval(e, f->mixed, f->s) != cudaSuccess) return GTAP_ERR_CUDA;
    cudaEventRecord(f->ev[7], f->s);
    if (cudaStreamSynchronize(f->s) != cudaSuccess) return GTAP_ERR_CUDA;
    f->info_h.ms_group = elapsed(f->ev[3], f->ev[4]);
    f->info_h.ms_m2l = elapsed(f->ev[4], f->ev[5]);
    f->info_h.ms_downward = elapsed(f->ev[5], f->ev[6]);
    f->info_h.ms_leaf = elapsed(f->ev[6], f->ev[7]);
    return GTAP_OK;
}

gtap_status gtap_fmm_run(gtap_fmm* f, gtap_ctx* ctx, const double* pos, const double* q, int64_t n, double* phi) {
    gtap_status st = gtap_fmm_build(f, pos, q, n);
    if (st == GTAP_OK) st = gtap_fmm_traverse(f, ctx);
    if (st == GTAP_OK) st = gtap_fmm_evaluate(f, phi);
    return st;
}

gtap_status gtap_fmm_get_info(const gtap_fmm* f, gtap_fmm_info* out) {
    if (!f || !out) return GTAP_ERR_INVALID_ARG;
    *out = f->info_h;
    out->n_points = f->n;
    out->n_cells = f->n_cells;
    out->n_leaves = f->n_leaves;
    out->n_levels = f->n_levels;
    out->order = f->p;
    out->n_m2l = f->n_m2l;
    out->n_p2p = f->n_p2p;
    out->m2l_capacity = f->m2l_cap;
    out->p2p_capacity = f->p2p_cap;
    return GTAP_OK;
}

gtap_status gtap_fmm_copy_tree(const gtap_fmm* f, int32_t* info, double* geom, int32_t* order) {
    if (!f || !f->built) return GTAP_ERR_INVALID_ARG;
    const size_t nc = (size_t)f->n_cells;
    if (info && cudaMemcpy(info, f->info.p, sizeof(int4) * nc, cudaMemcpyDeviceToHost) != cudaSuccess) return GTAP_ERR_CUDA;
    if (geom && cudaMemcpy(geom, f->geom.p, sizeof(Dbl4) * nc, cudaMemcpyDeviceToHost) != cudaSuccess)
        return GTAP_ERR_CUDA;
    if (order && cudaMemcpy(order, f->order, sizeof(uint32_t) * (size_t)f->n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return GTAP_ERR_CUDA;
    return GTAP_OK;
}

gtap_status gtap_fmm_copy_lists(const gtap_fmm* f, int32_t* m2l, int32_t* p2p) {
    if (!f || !f->built) return GTAP_ERR_INVALID_ARG;
    if (!f->traversed) return GTAP_ERR_LIST_OVERFLOW;
    struct Job { const DBuf* src; long long n; int32_t* dst; } jobs[2] = {{&f->m2l, f->n_m2l, m2l}, {&f->p2p, f->n_p2p, p2p}};
    for (const Job& j : jobs) {
        if (!j.dst || j.n == 0) continue;
        std::vector<unsigned long long> tmp((size_t)j.n);
        if (cudaMemcpy(tmp.data(), j.src->p, sizeof(unsigned long long) * tmp.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
            return GTAP_ERR_CUDA;
        for (size_t i = 0; i < tmp.size(); ++i) {
            j.dst[2 * i] = (int32_t)(tmp[i] >> 32);
            j.dst[2 * i + 1] = (int32_t)(tmp[i] & 0xFFFFFFFFull);
        }
    }
    return GTAP_OK;
}

gtap_status gtap_fmm_destroy(gtap_fmm* f) {
    if (!f) return GTAP_ERR_INVALID_ARG;
    cudaStreamSynchronize(f->s);
    delete f;
    return GTAP_OK;
}

}  // extern "C"
