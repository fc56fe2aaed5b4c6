"""CPU oracle for the fork-join workloads -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
(and its ``--impl reference`` arm) may import this package.  The library's
compute path never does: it shares no code with the oracle.

The routines live in ``oracle.cpp`` (plain sequential C++, serial elision of
each task program) and ``fmm_oracle.cpp`` (the FP64 Laplace FMM, stepwise);
this module builds them with g++ into ``liboracle.so`` and exposes thin ctypes
wrappers taking numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["oracle.cpp", "fmm_oracle.cpp"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no fused multiply-add, so every FP op rounds)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            u64, i64, i32, f64 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            P = ctypes.c_void_p
            sigs = {
                "orc_splitmix64_next": (u64, [u64]),
                "orc_fib": (i64, [i32, P]),
                "orc_nqueens_bitmask": (u64, [i32, P]),
                "orc_nqueens_array": (u64, [i32, P]),
                "orc_nqueens_permutations": (u64, [i32]),
                "orc_uts_recursive": (None, [u64, ctypes.c_uint32, ctypes.c_uint32, u64, P, P, P]),
                "orc_uts_bfs": (None, [u64, ctypes.c_uint32, ctypes.c_uint32, u64, P, P]),
                "orc_sort_u32": (None, [P, P, u64]),
                "orc_integrate_thread": (f64, [f64, f64, f64, P]),
                "orc_integrate_block": (f64, [f64, f64, f64, i32, P]),
                "orc_kclique": (u64, [i64, P, i64, i32, i32, P]),
                "orc_orient": (None, [i64, P, i64, i32, P, P]),
                "orc_kclique_brute": (u64, [i32, P, i64, i32]),
                "orc_kclique_edge_range": (u64, [i64, P, i64, i32, i32, i64, i64]),
                "orc_kclique_dag_ranges": (u64, [i64, P, P, i32, P, i64]),
                "orc_fmm": (i32, [i64, P, P, i32, f64, i32, P, i64, P, P, P, P, P, i64, P, i64]),
                "orc_fmm_tree": (i64, [i64, P, i32, P, i64, P]),
                "orc_direct": (None, [i64, P, P, P, i64, P]),
                "orc_taylor": (i32, [i32, f64, f64, f64, P]),
                "orc_bintree": (u64, [i32, i32, i32, i32, P]),
                "orc_fib_cutoff": (i64, [i32, i32, P]),
                "orc_cilksort": (u64, [P, P, u64, u64, u64]),
                "orc_kclique_pivot": (u64, [i64, P, i64, i32, i64, i64, P]),
                "orc_undirected": (None, [i64, P, i64, P, P]),
                "orc_kclique_pivot_all": (None, [i64, P, P, P, i64, i32, P]),
                "orc_nqueens_cutoff": (u64, [i32, i32, P]),
                "orc_bintree_leaf": (u64, [u64, i32, i32]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def splitmix64(state: int) -> int:
    return int(_load().orc_splitmix64_next(state))


def fib(n: int):
    """(fib(n), task count)."""
    t = ctypes.c_uint64(0)
    v = _load().orc_fib(n, ctypes.byref(t))
    return int(v), int(t.value)


def fib_cutoff(n: int, cutoff: int):
    """(fib(n), tasks) when calls below the cutoff run serially inside one leaf task."""
    t = ctypes.c_uint64(0)
    v = _load().orc_fib_cutoff(n, cutoff, ctypes.byref(t))
    return int(v), int(t.value)


def nqueens_cutoff(n: int, depth: int):
    """(solutions, tasks) when boards with `depth` rows placed finish their search serially."""
    t = ctypes.c_uint64(0)
    s = _load().orc_nqueens_cutoff(n, depth, ctypes.byref(t))
    return int(s), int(t.value)


def nqueens(n: int, algorithm: str = "bitmask"):
    """(solutions, tasks) for the one-task-per-placed-row N-Queens tree."""
    t = ctypes.c_uint64(0)
    fn = {"bitmask": _load().orc_nqueens_bitmask, "array": _load().orc_nqueens_array}[algorithm]
    s = fn(n, ctypes.byref(t))
    return int(s), int(t.value)


def nqueens_permutations(n: int) -> int:
    return int(_load().orc_nqueens_permutations(n))


UTS_THRESHOLD_Q0199 = 199 * 2 ** 64 // 1000  # floor(0.199 * 2^64), exact integer


def uts(seed: int = 42, root_children: int = 2000, m: int = 5, threshold: int = UTS_THRESHOLD_Q0199,
        algorithm: str = "recursive"):
    """(nodes, leaves) of the hashed unbalanced tree."""
    n, l, d = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    if algorithm == "recursive":
        _load().orc_uts_recursive(seed, root_children, m, threshold, ctypes.byref(n), ctypes.byref(l),
                                  ctypes.byref(d))
    else:
        _load().orc_uts_bfs(seed, root_children, m, threshold, ctypes.byref(n), ctypes.byref(l))
    return int(n.value), int(l.value)


def bintree(depth: int, iters: int, K: int = 1, cutoff: int = 0):
    """(sum of leaf values mod 2^64, tasks) of the full binary task tree (Sec. 6.1, 6.2)."""
    t = ctypes.c_uint64(0)
    v = _load().orc_bintree(depth, iters, K, cutoff, ctypes.byref(t))
    return int(v), int(t.value)


def bintree_leaf(v: int, iters: int, K: int = 1) -> int:
    """Value of leaf v of the binary task tree."""
    return int(_load().orc_bintree_leaf(v, iters, K))


def sort_u32(keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    out = np.empty_like(keys)
    _load().orc_sort_u32(_ptr(keys), _ptr(out), keys.size)
    return out


def cilksort(keys: np.ndarray, sort_cutoff: int = 64, merge_cutoff: int = 256):
    """(sorted keys, tasks) of the thread-mode Cilksort recursion."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    out = np.empty_like(keys)
    t = _load().orc_cilksort(_ptr(keys), _ptr(out), keys.size, sort_cutoff, merge_cutoff)
    return out, int(t)


def integrate_thread(a: float, b: float, eps: float):
    t = ctypes.c_uint64(0)
    v = _load().orc_integrate_thread(a, b, eps, ctypes.byref(t))
    return float(v), int(t.value)


def integrate_block(a: float, b: float, eps: float, block_size: int):
    t = ctypes.c_uint64(0)
    v = _load().orc_integrate_block(a, b, eps, block_size, ctypes.byref(t))
    return float(v), int(t.value)


def kclique(n: int, edges: np.ndarray, k: int, order: str = "degree", per_edge: bool = False):
    """Total k-clique count (and per-DAG-edge counts if asked)."""
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    m = edges.shape[0]
    pe = np.zeros(max(m, 1), dtype=np.uint64) if per_edge else None
    total = _load().orc_kclique(n, _ptr(edges), m, k, {"degree": 0, "id": 1}[order],
                                _ptr(pe) if pe is not None else None)
    return (int(total), pe[:m]) if per_edge else int(total)


def kclique_pivot(n: int, edges: np.ndarray, k: int, lo: int = 0, hi: int | None = None):
    """(k-clique count, recursion nodes) by pivoting over DAG edges [lo, hi) (all by default)."""
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    m = edges.shape[0]
    nodes = ctypes.c_uint64(0)
    c = _load().orc_kclique_pivot(n, _ptr(edges), m, k, lo, m if hi is None else hi, ctypes.byref(nodes))
    return int(c), int(nodes.value)


def undirected(n: int, edges: np.ndarray):
    """(uoff, uadj): the undirected CSR with sorted lists."""
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    m = edges.shape[0]
    uoff = np.zeros(n + 1, dtype=np.int64)
    uadj = np.zeros(max(2 * m, 1), dtype=np.int32)
    _load().orc_undirected(n, _ptr(edges), m, _ptr(uoff), _ptr(uadj))
    return uoff, uadj[: 2 * m]


def kclique_pivot_all(off: np.ndarray, adj: np.ndarray, ranges, kmax: int):
    """Clique counts of every size (list indexed by size, 0..kmax) by pivoting over DAG-edge
    ranges of a graph oriented by `orient`."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    rg = np.ascontiguousarray(np.asarray(ranges, dtype=np.int64).reshape(-1, 2))
    out = np.zeros(kmax + 1, dtype=np.uint64)
    _load().orc_kclique_pivot_all(off.shape[0] - 1, _ptr(off), _ptr(adj), _ptr(rg), rg.shape[0], kmax, _ptr(out))
    return [int(x) for x in out]


def orient(n: int, edges: np.ndarray, order: str = "degree"):
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    m = edges.shape[0]
    off = np.zeros(n + 1, dtype=np.int64)
    adj = np.zeros(max(m, 1), dtype=np.int32)
    _load().orc_orient(n, _ptr(edges), m, {"degree": 0, "id": 1}[order], _ptr(off), _ptr(adj))
    return off, adj[:m]


def kclique_brute(n: int, edges: np.ndarray, k: int) -> int:
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    return int(_load().orc_kclique_brute(n, _ptr(edges), edges.shape[0], k))


def kclique_edge_range(n: int, edges: np.ndarray, k: int, lo: int, hi: int, order: str = "degree") -> int:
    """Sum of per-DAG-edge k-clique counts over DAG edges [lo, hi)."""
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    return int(_load().orc_kclique_edge_range(n, _ptr(edges), edges.shape[0], k, {"degree": 0, "id": 1}[order], lo, hi))


def kclique_dag_ranges(off: np.ndarray, adj: np.ndarray, k: int, ranges) -> int:
    """Sum of per-DAG-edge k-clique counts over several edge ranges [lo, hi) of a
    graph already oriented by `orient` (for timing a sample of a large graph)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    rg = np.ascontiguousarray(np.asarray(ranges, dtype=np.int64).reshape(-1, 2))
    return int(_load().orc_kclique_dag_ranges(off.shape[0] - 1, _ptr(off), _ptr(adj), k, _ptr(rg), rg.shape[0]))


def fmm(pos: np.ndarray, q: np.ndarray, p: int = 6, theta: float = 0.5, leaf_size: int = 64,
        lists: bool = False, targets=None):
    """FP64 FMM potentials (input order, or at ``targets`` only).  With ``lists``: also
    (m2l, p2p) as (k, 2) int64 arrays of (target cell, source cell) in traversal order,
    and the cell count."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = q.size
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    phi = np.zeros(n if tg is None else max(tg.size, 1), dtype=np.float64)
    nc, nm, npp = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    lib = _load()
    tp, tn = (None, 0) if tg is None else (_ptr(tg), tg.size)
    if lib.orc_fmm(n, _ptr(pos), _ptr(q), p, theta, leaf_size, tp, tn, _ptr(phi), ctypes.byref(nc),
                   ctypes.byref(nm), ctypes.byref(npp), None, 0, None, 0) != 0:
        raise ValueError("orc_fmm: invalid arguments")
    if tg is not None:
        phi = phi[:tg.size]
    if not lists:
        return phi
    m2l = np.zeros((max(nm.value, 1), 2), dtype=np.int64)
    p2p = np.zeros((max(npp.value, 1), 2), dtype=np.int64)
    lib.orc_fmm(n, _ptr(pos), _ptr(q), p, theta, leaf_size, tp, tn, _ptr(np.zeros_like(phi)), None, None, None,
                _ptr(m2l), nm.value, _ptr(p2p), npp.value)
    return phi, m2l[:nm.value], p2p[:npp.value], int(nc.value)


def fmm_tree(pos: np.ndarray, leaf_size: int = 64):
    """(cells, order): cells is (n_cells, 8) float64 rows (level, first, count,
    child_first, nchild, cx, cy, cz); order maps sorted position -> input index."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    order = np.zeros(n, dtype=np.int64)
    cap = max(16, 4 * n // max(leaf_size, 1) + 64)
    while True:
        cells = np.zeros((cap, 8), dtype=np.float64)
        nc = int(_load().orc_fmm_tree(n, _ptr(pos), leaf_size, _ptr(cells), cap, _ptr(order)))
        if nc <= cap:
            return cells[:nc], order
        cap = nc


def direct(pos: np.ndarray, q: np.ndarray, targets=None) -> np.ndarray:
    """phi_i = sum_{j != i} q_j / |x_i - x_j| for the given targets (all by default)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = q.size
    t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    out = np.zeros(t.size, dtype=np.float64)
    _load().orc_direct(n, _ptr(pos), _ptr(q), _ptr(t), t.size, _ptr(out))
    return out


def multi_indices(p: int):
    """Multi-indices (a, b, c) of degree <= p in the expansions' order."""
    return [(a, b, k - a - b) for k in range(p + 1) for a in range(k, -1, -1) for b in range(k - a, -1, -1)]


def taylor(p: int, r) -> np.ndarray:
    """T_n(r) = d^n(1/|r|)/n! for |n| <= p, ordered as multi_indices(p)."""
    out = np.zeros(len(multi_indices(p)), dtype=np.float64)
    if _load().orc_taylor(p, float(r[0]), float(r[1]), float(r[2]), _ptr(out)) != 0:
        raise ValueError("orc_taylor: order out of range")
    return out
