"""Python binding of the C ABI in include/gtap.h (ctypes; argument marshalling only).

Every function here has the name of the C entry point it calls and does no
work of its own: the fork-join runtime runs entirely in libgtap.so.  A
non-zero status raises GtapError.  If the native library is missing this
module raises at import time: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgtap.so")

GTAP_MODE_THREAD = 0
GTAP_MODE_BLOCK = 1
GTAP_STEAL_FILL = 0
GTAP_STEAL_EMPTY = 1
GTAP_STEAL_HALF = 2
GTAP_STEAL_ONE = 4
GTAP_SCHED_BATCHED = 0
GTAP_SCHED_GLOBAL = 1
GTAP_SCHED_SINGLE = 2
GTAP_KCLIQUE_ORIENT = 0
GTAP_KCLIQUE_PIVOT = 1

STATUS = {
    0: "GTAP_OK", 1: "GTAP_ERR_INVALID_ARG", 2: "GTAP_ERR_NO_MEMORY", 3: "GTAP_ERR_POOL_EXHAUSTED",
    4: "GTAP_ERR_DEQUE_OVERFLOW", 5: "GTAP_ERR_LIST_OVERFLOW", 6: "GTAP_ERR_TIMEOUT", 7: "GTAP_ERR_CUDA",
    8: "GTAP_ERR_BUSY", 9: "GTAP_ERR_UNKNOWN_TASK", 10: "GTAP_ERR_TASK_FAILED", 11: "GTAP_ERR_NOT_READY",
}
globals().update({v: k for k, v in STATUS.items()})


class GtapError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class gtap_config(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int), ("threads_per_block", ctypes.c_int),
                ("deque_capacity", ctypes.c_int), ("steal_policy", ctypes.c_int), ("max_roots", ctypes.c_int),
                ("frame_bytes", ctypes.c_int), ("device_arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t),
                ("stream", ctypes.c_void_p), ("timeout_ns", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("scratch_bytes", ctypes.c_size_t), ("grid_blocks", ctypes.c_int), ("debug_checks", ctypes.c_int),
                ("scheduler", ctypes.c_int), ("idle_backoff_ns", ctypes.c_int)]


class gtap_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "tasks_executed", "tasks_created", "steps", "pops", "popped", "steal_attempts", "steals", "stolen",
        "idle_iterations", "pushes", "pushed", "frames_high_water", "scratch_used")] + [
        ("n_workers", ctypes.c_int), ("grid_blocks", ctypes.c_int), ("threads_per_block", ctypes.c_int),
        ("kernel_ms", ctypes.c_float), ("run_ms", ctypes.c_float)] + [
        (n, ctypes.c_uint64) for n in ("cycles_pop", "cycles_steal", "cycles_exec", "cycles_push", "cycles_idle")]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class gtap_error_info(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int), ("task_type", ctypes.c_int), ("worker", ctypes.c_int),
                ("pad", ctypes.c_int), ("detail", ctypes.c_uint64)]


class gtap_fib_args(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("route", ctypes.c_int32), ("cutoff", ctypes.c_int32), ("pad", ctypes.c_int32)]


class gtap_nqueens_args(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("route", ctypes.c_int32), ("cutoff", ctypes.c_int32), ("pad", ctypes.c_int32)]


class gtap_uts_args(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("threshold", ctypes.c_uint64), ("root_children", ctypes.c_uint32),
                ("m", ctypes.c_uint32), ("route", ctypes.c_int32), ("pad", ctypes.c_int32)]


class gtap_integrate_args(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("eps", ctypes.c_double)]


class gtap_kclique_args(ctypes.Structure):
    _fields_ = [("off", ctypes.c_void_p), ("adj", ctypes.c_void_p), ("src", ctypes.c_void_p),
                ("edge_begin", ctypes.c_int64), ("edge_end", ctypes.c_int64), ("k", ctypes.c_int32),
                ("split_threshold", ctypes.c_int32), ("route", ctypes.c_int32), ("algorithm", ctypes.c_int32)]


class gtap_bintree_args(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("iters", ctypes.c_int32), ("K", ctypes.c_int32), ("route", ctypes.c_int32),
                ("cutoff", ctypes.c_int32), ("pad", ctypes.c_int32)]


class gtap_cilksort_args(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("tmp", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("sort_cutoff", ctypes.c_uint32), ("merge_cutoff", ctypes.c_uint32), ("route", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class gtap_mergesort_args(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("tmp", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("leaf", ctypes.c_uint32), ("merge_cutoff", ctypes.c_uint32)]


class gtap_fmm_config(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("leaf_size", ctypes.c_int), ("theta", ctypes.c_double),
                ("precision", ctypes.c_int), ("fp64_levels", ctypes.c_int), ("m2l_capacity", ctypes.c_int64),
                ("p2p_capacity", ctypes.c_int64), ("stream", ctypes.c_void_p)]


class gtap_fmm_info(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_levels", ctypes.c_int), ("order", ctypes.c_int), ("n_m2l", ctypes.c_int64),
                ("n_p2p", ctypes.c_int64), ("m2l_capacity", ctypes.c_int64), ("p2p_capacity", ctypes.c_int64)] + [
        (n, ctypes.c_float) for n in ("ms_tree", "ms_upward", "ms_traverse", "ms_group", "ms_m2l", "ms_downward",
                                      "ms_leaf")]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class gtap_fmm_dtt_args(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("target", ctypes.c_int32), ("source", ctypes.c_int32)]


GTAP_FMM_FP64 = 0
GTAP_FMM_MIXED = 1


class gtap_tune_trial(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int), ("deque_capacity", ctypes.c_int), ("n_queues", ctypes.c_int),
                ("steal_policy", ctypes.c_int), ("kernel_ms", ctypes.c_float), ("status", ctypes.c_int),
                ("idle_backoff_ns", ctypes.c_int), ("pad", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad"}


class gtap_completion(ctypes.Structure):
    _fields_ = [("req", ctypes.c_uint64), ("result", ctypes.c_uint64 * 2), ("status", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


_P = ctypes.c_void_p
_SIGS = {
    "gtap_init": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(gtap_config),
                                 ctypes.POINTER(_P)]),
    "gtap_register_task": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]),
    "gtap_spawn_root": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "gtap_run": (ctypes.c_int, [_P]),
    "gtap_wait": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "gtap_read_result": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_size_t]),
    "gtap_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(gtap_stats)]),
    "gtap_last_error": (ctypes.c_int, [_P, ctypes.POINTER(gtap_error_info)]),
    "gtap_clear_roots": (ctypes.c_int, [_P]),
    "gtap_set_timeout": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "gtap_arena_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(gtap_config),
                                        ctypes.POINTER(ctypes.c_size_t)]),
    "gtap_capture_graph": (ctypes.c_int, [_P]),
    "gtap_serve_start": (ctypes.c_int, [_P]),
    "gtap_microbench": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double), _P]),
    "gtap_submit": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
    "gtap_poll": (ctypes.c_int, [_P, ctypes.POINTER(gtap_completion), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gtap_serve_stop": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "gtap_serve_progress": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]),
    "gtap_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gtap_finalize": (ctypes.c_int, [_P]),
    "gtap_debug_snapshot": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]),
    "gtap_mergesort_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_uint64, _P]),
    "gtap_kclique_orient": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, _P]),
    "gtap_fmm_create": (ctypes.c_int, [ctypes.POINTER(gtap_fmm_config), ctypes.POINTER(_P)]),
    "gtap_fmm_build": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64]),
    "gtap_fmm_traverse": (ctypes.c_int, [_P, _P]),
    "gtap_fmm_evaluate": (ctypes.c_int, [_P, _P]),
    "gtap_fmm_run": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P]),
    "gtap_fmm_get_info": (ctypes.c_int, [_P, ctypes.POINTER(gtap_fmm_info)]),
    "gtap_fmm_copy_tree": (ctypes.c_int, [_P, _P, _P, _P]),
    "gtap_fmm_copy_lists": (ctypes.c_int, [_P, _P, _P]),
    "gtap_fmm_destroy": (ctypes.c_int, [_P]),
    "gtap_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.c_char_p, _P, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_size_t, ctypes.POINTER(gtap_config), ctypes.c_int, ctypes.c_int, _P,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(gtap_tune_trial)]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgtap.so (build it first with paper_2604_05982_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"native library not built: {path} (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int, where: str, ok=(0,)):
    if status not in ok:
        raise GtapError(status, where)
    return status


def gtap_status_string(status: int) -> str:
    return load_library().gtap_status_string(status).decode()


def gtap_init(mode: int, n_queues: int, frame_pool_bytes: int, cfg: gtap_config | None = None) -> int:
    ctx = _P()
    _check(load_library().gtap_init(mode, n_queues, frame_pool_bytes, ctypes.byref(cfg) if cfg else None,
                                    ctypes.byref(ctx)), "gtap_init")
    return ctx.value


def gtap_register_task(ctx: int, program: str) -> int:
    t = ctypes.c_int(0)
    _check(load_library().gtap_register_task(ctx, program.encode(), ctypes.byref(t)), "gtap_register_task")
    return t.value


def gtap_spawn_root(ctx: int, type_id: int, args: ctypes.Structure, queue: int = 0) -> int:
    h = ctypes.c_uint64(0)
    _check(load_library().gtap_spawn_root(ctx, type_id, ctypes.byref(args), ctypes.sizeof(args), queue,
                                          ctypes.byref(h)), "gtap_spawn_root")
    return h.value


def gtap_run(ctx: int) -> None:
    _check(load_library().gtap_run(ctx), "gtap_run")


def gtap_wait(ctx: int, timeout_ms: int = 0, raise_on_error: bool = True) -> int:
    s = load_library().gtap_wait(ctx, timeout_ms)
    if raise_on_error:
        _check(s, "gtap_wait")
    return s


def gtap_read_result(ctx: int, handle: int, nbytes: int = 8) -> bytes:
    buf = (ctypes.c_char * nbytes)()
    _check(load_library().gtap_read_result(ctx, handle, buf, nbytes), "gtap_read_result")
    return bytes(buf)


def gtap_get_stats(ctx: int) -> gtap_stats:
    st = gtap_stats()
    _check(load_library().gtap_get_stats(ctx, ctypes.byref(st)), "gtap_get_stats")
    return st


def gtap_last_error(ctx: int) -> gtap_error_info:
    e = gtap_error_info()
    _check(load_library().gtap_last_error(ctx, ctypes.byref(e)), "gtap_last_error")
    return e


def gtap_clear_roots(ctx: int) -> None:
    _check(load_library().gtap_clear_roots(ctx), "gtap_clear_roots")


def gtap_set_timeout(ctx: int, timeout_ns: int) -> None:
    """Device-side deadline of later runs (0: the default of 60 s)."""
    _check(load_library().gtap_set_timeout(ctx, timeout_ns), "gtap_set_timeout")


def gtap_arena_bytes(mode: int, n_queues: int, frame_pool_bytes: int, cfg: gtap_config | None = None) -> int:
    """Device bytes gtap_init needs for these arguments (the size of a caller-owned arena)."""
    out = ctypes.c_size_t(0)
    _check(load_library().gtap_arena_bytes(mode, n_queues, frame_pool_bytes, ctypes.byref(cfg) if cfg else None,
                                           ctypes.byref(out)), "gtap_arena_bytes")
    return out.value


def gtap_capture_graph(ctx: int) -> None:
    _check(load_library().gtap_capture_graph(ctx), "gtap_capture_graph")


def gtap_finalize(ctx: int) -> None:
    _check(load_library().gtap_finalize(ctx), "gtap_finalize")


def gtap_debug_snapshot(ctx: int) -> dict:
    buf = (ctypes.c_uint64 * 9)()
    _check(load_library().gtap_debug_snapshot(ctx, buf, 9), "gtap_debug_snapshot")
    names = ["roots_remaining", "bump", "cq_enq", "cq_deq", "queued", "nonempty_queues", "locks_held",
             "max_count", "abort"]
    return dict(zip(names, list(buf)))


def gtap_mergesort_noalloc(src: int, dst: int, n: int, stream: int = 0, raise_on_error: bool = True) -> int:
    """Sort n uint32 keys (device pointers) without any device allocation; returns the status."""
    s = load_library().gtap_mergesort_noalloc(src, dst, n, stream or None)
    if raise_on_error:
        _check(s, "gtap_mergesort_noalloc")
    return s


def gtap_kclique_orient(edges: int, m: int, n: int, off: int, adj: int, src: int, work: int, stream: int = 0) -> None:
    """Orient an undirected graph on the GPU (device pointers; see gtap.h)."""
    _check(load_library().gtap_kclique_orient(edges, m, n, off, adj, src, work, stream or None), "gtap_kclique_orient")


def gtap_serve_start(ctx: int) -> None:
    _check(load_library().gtap_serve_start(ctx), "gtap_serve_start")


def gtap_submit(ctx: int, type_id: int, args: ctypes.Structure, queue: int = 0):
    """Queue a request; returns its id, or None if the inbox is full (GTAP_ERR_BUSY)."""
    r = ctypes.c_uint64(0)
    s = load_library().gtap_submit(ctx, type_id, ctypes.byref(args), ctypes.sizeof(args), queue, ctypes.byref(r))
    if s == GTAP_ERR_BUSY:
        return None
    _check(s, "gtap_submit")
    return r.value


_poll_buf = (gtap_completion * 4096)()


def gtap_poll(ctx: int, max_n: int = 4096):
    """Completed requests as (req, result0, result1, status) tuples."""
    n = ctypes.c_int(0)
    max_n = min(max_n, len(_poll_buf))
    _check(load_library().gtap_poll(ctx, _poll_buf, max_n, ctypes.byref(n)), "gtap_poll")
    return [(c.req, c.result[0], c.result[1], c.status) for c in _poll_buf[: n.value]]


def gtap_serve_progress(ctx: int):
    """(submitted, admitted by the device, completions polled)."""
    buf = (ctypes.c_uint64 * 3)()
    _check(load_library().gtap_serve_progress(ctx, buf, 3), "gtap_serve_progress")
    return tuple(int(x) for x in buf)


def gtap_serve_stop(ctx: int, timeout_ms: int = 0) -> int:
    s = load_library().gtap_serve_stop(ctx, timeout_ms)
    _check(s, "gtap_serve_stop")
    return s


MICROBENCH_KINDS = {0: "scattered acq_rel atomic add (join decrement)", 1: "scattered red.add u64 (accumulate)",
                    2: "per-warp CAS (deque claim)", 3: "single-word CAS (hot word)", 4: "scattered L2 load"}


def gtap_microbench(kind: int, region: int, region_bytes: int, blocks: int, threads: int = 256, iters: int = 64,
                    stream: int = 0):
    """Returns (ms, ops) of one timed launch."""
    ms = ctypes.c_float(0)
    ops = ctypes.c_double(0)
    _check(load_library().gtap_microbench(kind, region, region_bytes, blocks, threads, iters, ctypes.byref(ms),
                                          ctypes.byref(ops), stream or None), "gtap_microbench")
    return ms.value, ops.value


def gtap_fmm_create(cfg: gtap_fmm_config | None = None) -> int:
    f = _P()
    _check(load_library().gtap_fmm_create(ctypes.byref(cfg) if cfg else None, ctypes.byref(f)), "gtap_fmm_create")
    return f.value


def gtap_fmm_build(f: int, pos: int, q: int, n: int) -> None:
    _check(load_library().gtap_fmm_build(f, pos, q, n), "gtap_fmm_build")


def gtap_fmm_traverse(f: int, ctx: int) -> None:
    _check(load_library().gtap_fmm_traverse(f, ctx), "gtap_fmm_traverse")


def gtap_fmm_evaluate(f: int, phi: int) -> None:
    _check(load_library().gtap_fmm_evaluate(f, phi), "gtap_fmm_evaluate")


def gtap_fmm_run(f: int, ctx: int, pos: int, q: int, n: int, phi: int) -> None:
    _check(load_library().gtap_fmm_run(f, ctx, pos, q, n, phi), "gtap_fmm_run")


def gtap_fmm_get_info(f: int) -> gtap_fmm_info:
    out = gtap_fmm_info()
    _check(load_library().gtap_fmm_get_info(f, ctypes.byref(out)), "gtap_fmm_get_info")
    return out


def gtap_fmm_copy_tree(f: int, info, geom, order) -> None:
    """Host numpy outputs (int32 [n_cells, 4], float64 [n_cells, 4], int32 [n]); any may be None."""
    ptr = (lambda a: None if a is None else a.ctypes.data_as(_P))
    _check(load_library().gtap_fmm_copy_tree(f, ptr(info), ptr(geom), ptr(order)), "gtap_fmm_copy_tree")


def gtap_fmm_copy_lists(f: int, m2l, p2p) -> None:
    """Host numpy outputs (int32 [n_m2l, 2], int32 [n_p2p, 2]); either may be None."""
    ptr = (lambda a: None if a is None else a.ctypes.data_as(_P))
    _check(load_library().gtap_fmm_copy_lists(f, ptr(m2l), ptr(p2p)), "gtap_fmm_copy_lists")


def gtap_fmm_destroy(f: int) -> None:
    _check(load_library().gtap_fmm_destroy(f), "gtap_fmm_destroy")


GTAP_TUNE_BLOCKS, GTAP_TUNE_STEAL, GTAP_TUNE_QUEUES, GTAP_TUNE_CAPACITY, GTAP_TUNE_BACKOFF = 1, 2, 4, 8, 16


def gtap_autotune(mode: int, program: str, root_args, frame_pool_bytes: int, base: gtap_config | None = None,
                  reps: int = 3, max_trials: int = 64, n_queues: int = 1, tune_mask: int = 0):
    """Tune one program over a batch of roots (a list of args structs); returns (best, trials)."""
    root_args = list(root_args)
    n = len(root_args)
    size = ctypes.sizeof(root_args[0])
    buf = (ctypes.c_char * (size * n))()
    for i, a in enumerate(root_args):
        ctypes.memmove(ctypes.addressof(buf) + i * size, ctypes.addressof(a), size)
    trials = (gtap_tune_trial * max_trials)()
    nt = ctypes.c_int(0)
    best = gtap_tune_trial()
    _check(load_library().gtap_autotune(mode, program.encode(), buf, size, n, n_queues, frame_pool_bytes,
                                        ctypes.byref(base) if base else None, reps, tune_mask, trials, max_trials,
                                        ctypes.byref(nt), ctypes.byref(best)), "gtap_autotune")
    return best.as_dict(), [trials[i].as_dict() for i in range(min(nt.value, max_trials))]
