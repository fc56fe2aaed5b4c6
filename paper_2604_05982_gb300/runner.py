"""Convenience calls over the C ABI: one context, one batch of roots, one run.

Marshalling only: each helper creates a context (gtap_init), registers the
program, queues roots, runs, waits and reads results back.  All compute runs
in libgtap.so.
"""
from __future__ import annotations

import ctypes
import struct
from dataclasses import dataclass, field

from . import gtap as G

UTS_THRESHOLD_Q0199 = 199 * 2 ** 64 // 1000   # floor(0.199 * 2^64)


@dataclass
class RunResult:
    values: list
    stats: dict = field(default_factory=dict)
    status: int = 0


DEFAULT_TIMEOUT_NS = 20 * 10 ** 9   # device-side deadline of a helper run


def make_config(**kw) -> G.gtap_config:
    cfg = G.gtap_config()
    cfg.timeout_ns = DEFAULT_TIMEOUT_NS
    for k, v in kw.items():
        if v is not None:
            setattr(cfg, k, v)
    return cfg


class Context:
    """RAII wrapper of a gtap context (marshalling only)."""

    def __init__(self, mode: int, n_queues: int = 1, pool_bytes: int = 1 << 30, **cfg):
        self.cfg = make_config(**cfg)
        self.ctx = G.gtap_init(mode, n_queues, pool_bytes, self.cfg)

    def register(self, program: str) -> int:
        return G.gtap_register_task(self.ctx, program)

    def spawn(self, type_id: int, args, queue: int = 0) -> int:
        return G.gtap_spawn_root(self.ctx, type_id, args, queue)

    def run(self, timeout_ms: int = 0, raise_on_error: bool = True) -> int:
        G.gtap_run(self.ctx)
        return G.gtap_wait(self.ctx, timeout_ms, raise_on_error)

    def result_u64(self, h: int) -> int:
        return struct.unpack("<Q", G.gtap_read_result(self.ctx, h, 8))[0]

    def result_i64(self, h: int) -> int:
        return struct.unpack("<q", G.gtap_read_result(self.ctx, h, 8))[0]

    def result_f64(self, h: int) -> float:
        return struct.unpack("<d", G.gtap_read_result(self.ctx, h, 8))[0]

    def stats(self) -> dict:
        return G.gtap_get_stats(self.ctx).as_dict()

    def last_error(self) -> G.gtap_error_info:
        return G.gtap_last_error(self.ctx)

    def clear(self):
        G.gtap_clear_roots(self.ctx)

    def capture(self):
        G.gtap_capture_graph(self.ctx)

    def close(self):
        if self.ctx:
            G.gtap_finalize(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fib(ns, n_queues: int = 1, route: int = 0, cutoff: int = 0, **cfg) -> RunResult:
    ns = [ns] if isinstance(ns, int) else list(ns)
    with Context(G.GTAP_MODE_THREAD, n_queues, **cfg) as c:
        t = c.register("fib")
        hs = [c.spawn(t, G.gtap_fib_args(n, route, cutoff, 0)) for n in ns]
        c.run()
        return RunResult([c.result_i64(h) for h in hs], c.stats())


def nqueens(ns, n_queues: int = 1, route: int = 0, cutoff: int = 0, **cfg) -> RunResult:
    ns = [ns] if isinstance(ns, int) else list(ns)
    with Context(G.GTAP_MODE_THREAD, n_queues, **cfg) as c:
        t = c.register("nqueens")
        hs = [c.spawn(t, G.gtap_nqueens_args(n, route, cutoff, 0)) for n in ns]
        c.run()
        return RunResult([c.result_u64(h) for h in hs], c.stats())


def uts(seed: int = 42, root_children: int = 2000, m: int = 5, threshold: int = UTS_THRESHOLD_Q0199,
        n_queues: int = 1, route: int = 0, **cfg) -> RunResult:
    """Result values: [(nodes, leaves)]."""
    with Context(G.GTAP_MODE_THREAD, n_queues, **cfg) as c:
        t = c.register("uts")
        h = c.spawn(t, G.gtap_uts_args(seed, threshold, root_children, m, route, 0))
        c.run()
        v = c.result_u64(h)
        return RunResult([(v >> 32, v & 0xFFFFFFFF)], c.stats())


def bintree(depth: int, iters: int, K: int = 1, route: int = 0, block: bool = False, cutoff: int = 0,
            n_queues: int = 1, **cfg) -> RunResult:
    """Full binary task tree (Sec. 6.1, 6.2): thread mode ("bintree") or block mode ("bintree_block")."""
    mode = G.GTAP_MODE_BLOCK if block else G.GTAP_MODE_THREAD
    with Context(mode, n_queues, **cfg) as c:
        t = c.register("bintree_block" if block else "bintree")
        h = c.spawn(t, G.gtap_bintree_args(depth, iters, K, route, cutoff, 0))
        c.run()
        return RunResult([c.result_u64(h)], c.stats())


def integrate(a: float, b: float, eps: float, block: bool = False, **cfg) -> RunResult:
    mode = G.GTAP_MODE_BLOCK if block else G.GTAP_MODE_THREAD
    with Context(mode, 1, **cfg) as c:
        t = c.register("integrate_block" if block else "integrate")
        h = c.spawn(t, G.gtap_integrate_args(a, b, eps))
        c.run()
        return RunResult([c.result_f64(h)], c.stats())


def mergesort_ptrs(src: int, dst: int, tmp: int, n: int, leaf: int = 4096, merge_cutoff: int = 4096,
                   **cfg) -> RunResult:
    """Sort n uint32 keys at device address src into dst (tmp: n-key scratch)."""
    with Context(G.GTAP_MODE_BLOCK, 1, pool_bytes=256 << 20, **cfg) as c:
        t = c.register("mergesort")
        c.spawn(t, G.gtap_mergesort_args(src, dst, tmp, n, leaf, merge_cutoff))
        c.run()
        return RunResult([], c.stats())


def cilksort_ptrs(src: int, dst: int, tmp: int, n: int, sort_cutoff: int = 64, merge_cutoff: int = 256,
                  n_queues: int = 1, route: int = 0, **cfg) -> RunResult:
    """Thread-mode Cilksort of n uint32 keys at device address src into dst (tmp: n-key scratch)."""
    with Context(G.GTAP_MODE_THREAD, n_queues, **cfg) as c:
        t = c.register("cilksort")
        c.spawn(t, G.gtap_cilksort_args(src, dst, tmp, n, sort_cutoff, merge_cutoff, route, 0))
        c.run()
        return RunResult([], c.stats())


class DeviceGraph:
    """An undirected graph oriented on the GPU (gtap_kclique_orient); device buffers held as torch tensors."""

    def __init__(self, n: int, edges, stream: int = 0):
        import numpy as np
        import torch
        e = torch.as_tensor(np.ascontiguousarray(edges, dtype=np.int32)).reshape(-1, 2).cuda()
        m = int(e.shape[0])
        self.n, self.m = n, m
        self.edges = e
        self.off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        self.adj = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
        self.src = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
        self.work = torch.empty(4 * n + 16, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        G.gtap_kclique_orient(e.data_ptr(), m, n, self.off.data_ptr(), self.adj.data_ptr(), self.src.data_ptr(),
                              self.work.data_ptr(), stream)

    def args(self, k: int, split_threshold: int = 64, route: int = 0, begin: int = 0, end: int | None = None,
             algorithm: int = 0):
        return G.gtap_kclique_args(self.off.data_ptr(), self.adj.data_ptr(), self.src.data_ptr(), begin,
                                   self.m if end is None else end, k, split_threshold, route, algorithm)


def kclique(graphs, k: int, split_threshold: int = 64, n_queues: int = 1, route: int = 0,
            scratch_bytes: int = 1 << 30, ranges=None, algorithm: int = 0, **cfg) -> RunResult:
    """Count k-cliques of one or more DeviceGraphs in one persistent launch (one root each);
    algorithm 0: orientation, 1: pivoting."""
    graphs = [graphs] if isinstance(graphs, DeviceGraph) else list(graphs)
    with Context(G.GTAP_MODE_THREAD, n_queues, scratch_bytes=scratch_bytes, **cfg) as c:
        t = c.register("kclique")
        hs = []
        for i, g in enumerate(graphs):
            b, e = (0, g.m) if ranges is None else ranges[i]
            hs.append(c.spawn(t, g.args(k, split_threshold, route, b, e, algorithm), queue=0))
        c.run()
        return RunResult([c.result_u64(h) for h in hs], c.stats())


class Fmm:
    """A Laplace FMM plan plus the block-mode context its traversal runs on (marshalling only).

    ``run(pos, q)`` takes host or CUDA arrays (n x 3 and n, FP64) and returns the
    potentials as a CUDA float64 tensor in input order.  The traversal context
    defaults to 6 resident blocks of 128 threads per SM, what its kernel's
    registers allow (N = 2^20: 1.48 -> 1.20 ms uniform, 4.09 -> 3.27 ms Plummer
    against 4 blocks)."""

    def __init__(self, order: int = 6, leaf_size: int = 64, theta: float = 0.5, mixed: bool = False,
                 fp64_levels: int = 3, threads_per_block: int = 128, pool_bytes: int = 1 << 30,
                 deque_capacity: int = 4096, blocks_per_sm: int = 6, **cfg):
        fc = G.gtap_fmm_config()
        fc.order, fc.leaf_size, fc.theta = order, leaf_size, theta
        fc.precision = G.GTAP_FMM_MIXED if mixed else G.GTAP_FMM_FP64
        fc.fp64_levels = fp64_levels
        self.plan = G.gtap_fmm_create(fc)
        self.ctx = Context(G.GTAP_MODE_BLOCK, 1, pool_bytes=pool_bytes, threads_per_block=threads_per_block,
                           deque_capacity=deque_capacity, blocks_per_sm=blocks_per_sm, **cfg)

    def build(self, pos, q):
        import torch
        self.pos = torch.as_tensor(pos, dtype=torch.float64).reshape(-1, 3).contiguous().cuda()
        self.q = torch.as_tensor(q, dtype=torch.float64).reshape(-1).contiguous().cuda()
        self.n = int(self.q.shape[0])
        torch.cuda.synchronize()
        G.gtap_fmm_build(self.plan, self.pos.data_ptr(), self.q.data_ptr(), self.n)

    def traverse(self):
        G.gtap_fmm_traverse(self.plan, self.ctx.ctx)

    def evaluate(self):
        import torch
        phi = torch.empty(self.n, dtype=torch.float64, device="cuda")
        G.gtap_fmm_evaluate(self.plan, phi.data_ptr())
        return phi

    def run(self, pos, q):
        self.build(pos, q)
        self.traverse()
        return self.evaluate()

    def info(self) -> dict:
        return G.gtap_fmm_get_info(self.plan).as_dict()

    def tree(self):
        import numpy as np
        inf = self.info()
        nc = int(inf["n_cells"])
        info = np.zeros((nc, 4), dtype=np.int32)
        geom = np.zeros((nc, 4), dtype=np.float64)
        order = np.zeros(self.n, dtype=np.int32)
        G.gtap_fmm_copy_tree(self.plan, info, geom, order)
        return info, geom, order

    def lists(self):
        import numpy as np
        inf = self.info()
        m2l = np.zeros((int(inf["n_m2l"]), 2), dtype=np.int32)
        p2p = np.zeros((int(inf["n_p2p"]), 2), dtype=np.int32)
        G.gtap_fmm_copy_lists(self.plan, m2l, p2p)
        return m2l, p2p

    def close(self):
        if self.plan:
            G.gtap_fmm_destroy(self.plan)
            self.plan = None
        self.ctx.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
