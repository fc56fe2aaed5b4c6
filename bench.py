"""Benchmark of the fork-join runtime on the integer workload set of the paper's evaluation.

One step = one pass of the three workloads of the integer benchmark set,
each one persistent-kernel run through the C ABI:
  * N-Queens n=13, thread mode, one task per placed row, DAQ with 4 queues
    routed by depth mod 4 (4,674,890 tasks);
  * the unbalanced hashed tree, seed 42, root 2000 children, m=5, q=0.199
    (173,496 node tasks);
  * block-mode mergesort of 2^26 uniform uint32 keys, 4096-key leaves
    (32,767 sort tasks in the recursion tree; merges fork further pieces).
metric: tasks/s = (N-Queens nodes + tree nodes + sort-tree tasks) per second.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on
the host cores for the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NQ_N = 13
NQ_TASKS = 4674890
UTS_NODES = 173496
MSORT_LOG2 = 26
MSORT_LEAF = 4096
MSORT_SORT_TASKS = 2 * ((1 << MSORT_LOG2) // MSORT_LEAF) - 1
STEP_TASKS = NQ_TASKS + UTS_NODES + MSORT_SORT_TASKS
MSORT_BYTES = 8.05e9 * (1 << MSORT_LOG2) / (1 << 26)   # algorithmic HBM bytes: leaf pass + 14 merge levels

CONFIG = {"workload": "integer set: nqueens13 thread DAQ4 (depth mod 4) + hashed tree seed42 (2000, m=5, q=0.199) "
                      "+ block mergesort 2^26 u32 (4096-key leaves)",
          "nqueens_n": NQ_N, "tree_seed": 42, "mergesort_keys": 1 << MSORT_LOG2, "mergesort_leaf": MSORT_LEAF,
          "daq_queues": 4, "l2": "mergesort input 256 MiB > L2 (129 MB); task records re-initialised every run",
          "parallelism": "replicas"}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # a timed region shorter than the sampling period still gets a sample on
            # each side: wait for the first one here and for one more in __exit__
            t0 = time.perf_counter()
            while not self.samples and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            n0, t0 = len(self.samples), time.perf_counter()
            while len(self.samples) == n0 and time.perf_counter() - t0 < 1.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                mx = float(s[2])
                for name, v in zip(names, s[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value: float, device: str = "cuda") -> float:
    """Barrier, then the maximum of `value` over all ranks (one rank: the value itself)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def aggregate_rate(units_per_rank_step: float, steps: int, world: int, elapsed_ms: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank_step * steps * world / (elapsed_ms / 1e3)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2604_05982_gb300 import gtap as G
    from paper_2604_05982_gb300 import inputs, runner

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    G.load_library()

    n = 1 << MSORT_LOG2
    keys = inputs.keys_u32(n, seed=1)
    src = torch.from_numpy(keys.view(np.int32)).cuda()
    dst = torch.empty_like(src)
    tmp = torch.empty_like(src)
    torch.cuda.synchronize()

    nq_args = G.gtap_nqueens_args(NQ_N, 1)
    ut_args = G.gtap_uts_args(42, runner.UTS_THRESHOLD_Q0199, 2000, 5, 0, 0)
    ms_args = G.gtap_mergesort_args(src.data_ptr(), dst.data_ptr(), tmp.data_ptr(), n, MSORT_LEAF, 65536)
    # launch configuration per workload from the autotuner (outside the timed region); the
    # workload definitions stay fixed: N-Queens keeps its 4 DAQ queues, the others one queue
    tuned = {}
    tmask = G.GTAP_TUNE_BLOCKS | G.GTAP_TUNE_STEAL | G.GTAP_TUNE_CAPACITY | G.GTAP_TUNE_BACKOFF
    for key, mode, prog, a, q, pool in (("nqueens", G.GTAP_MODE_THREAD, "nqueens", nq_args, 4, 1 << 30),
                                        ("tree", G.GTAP_MODE_THREAD, "uts", ut_args, 1, 1 << 30),
                                        ("mergesort", G.GTAP_MODE_BLOCK, "mergesort", ms_args, 1, 256 << 20)):
        if args.no_tune:
            tuned[key] = {"blocks_per_sm": 4, "steal_policy": 0, "deque_capacity": 4096 if mode == 0 else 1024,
                          "idle_backoff_ns": 512}
        else:
            best, _ = G.gtap_autotune(mode, prog, [a], pool, runner.make_config(), reps=3, n_queues=q, tune_mask=tmask)
            tuned[key] = {k: best[k] for k in ("blocks_per_sm", "steal_policy", "deque_capacity", "idle_backoff_ns")}

    def ctx_for(key, mode, q, pool):
        c = tuned[key]
        return runner.Context(mode, q, pool_bytes=pool, blocks_per_sm=c["blocks_per_sm"],
                              steal_policy=c["steal_policy"], deque_capacity=c["deque_capacity"],
                              idle_backoff_ns=c["idle_backoff_ns"])

    nq = ctx_for("nqueens", G.GTAP_MODE_THREAD, 4, 1 << 30)
    t = nq.register("nqueens")
    h_nq = nq.spawn(t, nq_args)
    ut = ctx_for("tree", G.GTAP_MODE_THREAD, 1, 1 << 30)
    t = ut.register("uts")
    h_ut = ut.spawn(t, ut_args)
    ms = ctx_for("mergesort", G.GTAP_MODE_BLOCK, 1, 256 << 20)
    t = ms.register("mergesort")
    ms.spawn(t, ms_args)
    launches_per_step = 6   # each run: reset kernel + persistent scheduler kernel

    def step():
        t_nq = nq.run()
        t_ut = ut.run()
        t_ms = ms.run()
        return nq.stats()["kernel_ms"], ut.stats()["kernel_ms"], ms.stats()["kernel_ms"]

    for _ in range(args.warmup):
        step()
    # parity spot check of this exact launch configuration (outside the timed region)
    assert nq.result_u64(h_nq) == 73712
    v = ut.result_u64(h_ut)
    assert (v >> 32, v & 0xFFFFFFFF) == (UTS_NODES, 139196)
    out = dst[:: 1 << 12].cpu().numpy().view(np.uint32)
    assert np.all(out[1:] >= out[:-1])

    tasks_nq, tasks_ut = nq.stats()["tasks_created"], ut.stats()["tasks_created"]
    ceil = atomic_ceiling(local)
    per_kernel = {"nqueens": [], "tree": [], "mergesort": []}
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            a, b, c = step()
            per_kernel["nqueens"].append(a)
            per_kernel["tree"].append(b)
            per_kernel["mergesort"].append(c)
        e1.record()
        torch.cuda.synchronize()
    elapsed_ms = max_over_ranks(e0.elapsed_time(e1))
    ms_per_step = elapsed_ms / args.steps
    value = aggregate_rate(STEP_TASKS, args.steps, world, elapsed_ms)

    # end to end through the C ABI with host buffers: H2D of the keys from pinned memory,
    # the three runs, and D2H of the sorted keys and of the counts (gtap_wait reads them back)
    pinned_in = torch.from_numpy(keys.view(np.int32)).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record()
    for _ in range(args.steps):
        src.copy_(pinned_in, non_blocking=True)
        step()
        pinned_out.copy_(dst, non_blocking=True)
    e3.record()
    torch.cuda.synchronize()
    e2e_ms = e2.elapsed_time(e3) / args.steps

    hbm_peak, peak_kind = _peaks()
    ms_kernel = sorted(per_kernel["mergesort"])[len(per_kernel["mergesort"]) // 2]
    achieved = MSORT_BYTES / (ms_kernel / 1e3) / 1e9
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            traffic = json.load(f).get("mergesort_2pow26_bytes")
    except (OSError, ValueError):
        pass
    line = {
        "metric": "tasks/s", "value": value, "unit": "tasks/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic", "config": CONFIG,
        "breakdown_ms": {k: sorted(v)[len(v) // 2] for k, v in per_kernel.items()},
        "launch_config": {"source": "default" if args.no_tune else "gtap_autotune (blocks/SM, steal policy, idle "
                          "back-off, ring capacity; queue counts fixed by the workloads)", **tuned},
        "roofline": {"bound": "hbm", "kernel": "block_kernel<mergesort> (2^26 keys)", "achieved": achieved,
                     "peak": hbm_peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "traffic": traffic, "algorithmic_bytes": MSORT_BYTES},
        # every kernel of the step against its own ceiling: the sort against HBM, the two
        # thread-mode schedulers against the measured join-decrement rate (one acq_rel
        # decrement per non-root task)
        "rooflines": [
            {"bound": "hbm", "kernel": "block_kernel<mergesort>", "achieved": achieved, "peak": hbm_peak,
             "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic},
            _atomic_roofline("thread_kernel<nqueens> (DAQ 4)", tasks_nq, tasks_nq - 1, 0,
                             sorted(per_kernel["nqueens"])[len(per_kernel["nqueens"]) // 2], ceil),
            _atomic_roofline("thread_kernel<uts>", tasks_ut, tasks_ut - 1, 0,
                             sorted(per_kernel["tree"])[len(per_kernel["tree"]) // 2], ceil)],
        "atomic_ceiling_gops": {k: x / 1e9 for k, x in ceil.items()},
        "e2e": {"value": STEP_TASKS / (e2e_ms / 1e3), "unit": "tasks/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": n * 4 + 3 * 128, "d2h_bytes_per_step": n * 4 + 3 * 32},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    for c in (nq, ut, ms):
        c.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _cpu_step():
    """One bounded pass of the CPU oracle over the same workload (single thread)."""
    import oracle
    from paper_2604_05982_gb300 import inputs
    t0 = time.perf_counter()
    s, tasks = oracle.nqueens(NQ_N)
    assert (s, tasks) == (73712, NQ_TASKS)
    assert oracle.uts(42) == (UTS_NODES, 139196)
    keys = inputs.keys_u32(1 << MSORT_LOG2, seed=1)
    t1 = time.perf_counter()
    oracle.sort_u32(keys)
    t2 = time.perf_counter()
    return (t1 - t0) + (t2 - t1)


def cpu_baseline():
    import oracle
    oracle.build()
    try:
        os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    except (AttributeError, OSError):
        pass
    secs = _cpu_step()
    return {"value": STEP_TASKS / secs, "unit": "tasks/s", "cores": 1, "kind": "oracle",
            "sample": "one full step: oracle N-Queens(13), hashed tree seed 42, std::sort of the same 2^26 keys "
                      f"(single thread, {secs:.2f} s)"}


def run_reference_fmm(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    for _ in range(min(args.warmup, 1)):
        _fmm_cpu_sample()
    times = [_fmm_cpu_sample() for _ in range(args.steps)]
    secs = sum(times) / len(times)
    value = secs * 1e3 * FMM_N / FMM_CPU_SAMPLE_N
    line = {"impl": "reference", "metric": "FMM time", "value": value, "unit": "ms/instance", "n_gpus": world,
            "steps": args.steps, "warmup": min(args.warmup, 1), "ms_per_step": 2 * value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"Laplace FMM N=2^20, p={FMM_P}, theta={FMM_THETA}, leaf {FMM_LEAF} (oracle)"},
            "cpu_baseline": {"value": value, "unit": "ms/instance", "cores": 1, "kind": "oracle",
                             "sample": "oracle FMM on the first 2^16 uniform points per step, scaled x16"},
            "e2e": {"value": value, "unit": "ms/instance", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    if args.workload == "fmm":
        run_reference_fmm(args)
        return
    if args.workload == "kclique":
        run_reference_kclique(args)
        return
    if args.workload == "serve":
        run_reference_serve(args)
        return
    if args.workload in ("fib", "sched", "micro", "batch"):
        run_reference_small(args)
        return
    import oracle
    oracle.build()
    try:
        os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    except (AttributeError, OSError):
        pass
    for _ in range(args.warmup):
        _cpu_step()
    times = [_cpu_step() for _ in range(args.steps)]
    secs = sum(times)
    value = STEP_TASKS * args.steps / secs
    line = {"impl": "reference", "metric": "tasks/s", "value": value, "unit": "tasks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
            "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                             "sample": "full step per iteration, single thread"},
            "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_small(args):
    """Reference arm (the oracle on one host core) of the fib, sched, micro and batch lines."""
    import oracle
    oracle.build()
    _pin_one_core()
    world, _, _ = _dist()

    def sample():
        t0 = time.perf_counter()
        if args.workload in ("fib", "sched"):
            n = FIB_N if args.workload == "fib" else SCHED_N
            v, tasks = oracle.fib(n)
            return tasks, time.perf_counter() - t0
        if args.workload == "micro":
            oracle.bintree(16, 2048, 1)   # D = 16 of the D = 25 tree: 1/512 of the leaves
            return 1, (time.perf_counter() - t0) * 512
        from paper_2604_05982_gb300 import inputs
        graphs = [inputs.rmat_graph(12 + (7 * i) // 64, 16, seed=7 + i) for i in (0, 18, 27, 36)]
        t0 = time.perf_counter()
        for n, e in graphs:
            oracle.kclique(n, e, 4)
        return len(graphs), time.perf_counter() - t0

    for _ in range(min(args.warmup, 1)):
        sample()
    res = [sample() for _ in range(args.steps)]
    units = sum(r[0] for r in res)
    secs = sum(r[1] for r in res)
    if args.workload in ("fib", "sched"):
        n = FIB_N if args.workload == "fib" else SCHED_N
        metric, unit, value, hib = "tasks/s", "tasks/s", units / secs, True
        wl, note = f"fib({n}) thread mode (oracle)", f"oracle fib({n}) serial recursion per step"
    elif args.workload == "micro":
        metric, unit, value, hib = "binary-tree time", "ms", 1e3 * secs / args.steps, False
        wl, note = ("binary task tree D = 25, compute_iters 2048 (oracle)",
                    "oracle binary tree of depth 16 (1/512 of the leaves) per step, scaled x512")
    else:
        metric, unit, value, hib = "batched jobs/s", "instances/s", units / secs, True
        wl, note = ("batched 4-clique, 64 R-MAT graphs scales 12-18 (oracle)",
                    "oracle 4-clique count of graphs 0, 18, 27, 36 of the batch (scales 12-15) per step; "
                    "the larger graphs are slower, so this overstates the oracle's rate on the whole batch")
    line = {"impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": hib, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": wl},
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle", "sample": note},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


FMM_N = 1 << 20
FMM_P = 6
FMM_THETA = 0.5
FMM_LEAF = 64
FMM_SETS = ("uniform", "plummer")
FMM_CPU_SAMPLE_N = 1 << 16
FP32_LANES_PER_SM = 128     # FP32 FMA lanes per SM (GB300)
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64, nominal


def m2l_flops_per_pair(p: int) -> int:
    """Arithmetic of one M2L translation as the kernel performs it: the Taylor
    recurrence (3 flops per first-order term, 2 per second-order term, 1 for the
    final scaling, plus r^2, 1/r^2 and 1/r) and one FMA per (alpha, beta) term."""
    fl = 7
    for k in range(1, p + 1):
        for a in range(k, -1, -1):
            for b in range(k - a, -1, -1):
                n = (a, b, k - a - b)
                fl += 3 * sum(1 for x in n if x > 0) + 2 * sum(1 for x in n if x > 1) + 1
    terms = sum(1 for k1 in range(p + 1) for _ in range((k1 + 1) * (k1 + 2) // 2)
                for k2 in range(p - k1 + 1) for _ in range((k2 + 1) * (k2 + 2) // 2))
    return fl + 2 * terms


FMM_LEVEL_CHUNKS = (8, 12, 16, 21)   # the tree build checks for an empty level after these levels


def _fmm_levels_refined(n_levels: int) -> int:
    """Levels the tree build refines: up to the first chunk boundary at or past the
    first empty level (levels 0 .. n_levels-1 hold cells)."""
    return next((b for b in FMM_LEVEL_CHUNKS if b >= n_levels), FMM_LEVEL_CHUNKS[-1])


def _fmm_kernels_per_instance(n_levels: int, mixed: bool) -> int:
    done = _fmm_levels_refined(n_levels)
    # bbox (2), codes, 8 radix passes (histogram, 3-kernel scan, scatter), 5 kernels per refined level,
    # level-start tail when stopped early, gather, record check, leaf-local coordinates (mixed)
    tree = 2 + 1 + 8 * 5 + done * 5 + (1 if done < 21 else 0) + 1 + 1 + (1 if mixed else 0)
    upward = 1 + max(n_levels - 1, 0)
    traverse = 2
    evaluate = 2 * 5 + 2 + max(n_levels - 1, 0) + 1
    return tree + upward + traverse + evaluate


def run_fmm(args):
    import numpy as np
    import torch

    from paper_2604_05982_gb300 import gtap as G
    from paper_2604_05982_gb300 import inputs, runner
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    mixed = args.fmm_precision == "mixed"
    sets = {}
    for dist in FMM_SETS:
        pos, q = inputs.fmm_points(FMM_N, dist, seed=3)
        f = runner.Fmm(order=FMM_P, leaf_size=FMM_LEAF, theta=FMM_THETA, mixed=mixed)
        sets[dist] = dict(pos_h=pos, q_h=q, f=f, pos=torch.from_numpy(pos).cuda(), q=torch.from_numpy(q).cuda(),
                          phi=torch.empty(FMM_N, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()

    def instance(d):
        f = d["f"]
        G.gtap_fmm_build(f.plan, d["pos"].data_ptr(), d["q"].data_ptr(), FMM_N)
        G.gtap_fmm_traverse(f.plan, f.ctx.ctx)
        G.gtap_fmm_evaluate(f.plan, d["phi"].data_ptr())

    def step():
        for d in sets.values():
            instance(d)

    for _ in range(args.warmup):
        step()
    # parity spot check of this exact configuration (outside the timed region): 64 sampled
    # targets against the FP64 oracle FMM evaluated at those targets
    import oracle
    tg = np.arange(0, FMM_N, FMM_N // 64, dtype=np.int64)
    errs = {}
    for dist, d in sets.items():
        ref = oracle.fmm(d["pos_h"], d["q_h"], p=FMM_P, theta=FMM_THETA, leaf_size=FMM_LEAF, targets=tg)
        got = d["phi"].cpu().numpy()[tg]
        errs[dist] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert errs[dist] <= (1e-5 if mixed else 1e-12), errs
    phases = {dist: [] for dist in sets}
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            for dist, d in sets.items():
                instance(d)
                phases[dist].append(d["f"].info())
        e1.record()
        torch.cuda.synchronize()
    elapsed_ms = max_over_ranks(e0.elapsed_time(e1))
    ms_per_instance = elapsed_ms / (args.steps * len(sets) * world)

    # end to end through the public calls with host buffers: pinned H2D of positions and
    # charges, the three calls, D2H of the potentials
    pinned = {dist: (torch.from_numpy(d["pos_h"]).pin_memory(), torch.from_numpy(d["q_h"]).pin_memory(),
                     torch.empty(FMM_N, dtype=torch.float64).pin_memory()) for dist, d in sets.items()}
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record()
    for _ in range(args.steps):
        for dist, d in sets.items():
            ph, qh, out = pinned[dist]
            d["pos"].copy_(ph, non_blocking=True)
            d["q"].copy_(qh, non_blocking=True)
            instance(d)
            out.copy_(d["phi"], non_blocking=True)
    e3.record()
    torch.cuda.synchronize()
    e2e_ms = e2.elapsed_time(e3) / (args.steps * len(sets))

    def med(dist, key):
        v = sorted(x[key] for x in phases[dist])
        return v[len(v) // 2]

    keys = ("ms_tree", "ms_upward", "ms_traverse", "ms_group", "ms_m2l", "ms_downward", "ms_leaf")
    breakdown = {dist: {k: med(dist, k) for k in keys} for dist in sets}
    info = {dist: phases[dist][-1] for dist in sets}
    # roofline of the dominant kernel (M2L): ALU bound, peak from unit counts and the maximum clock
    fl = m2l_flops_per_pair(FMM_P)
    pairs = sum(info[dd]["n_m2l"] for dd in sets)
    m2l_ms = sum(breakdown[dd]["ms_m2l"] for dd in sets)
    achieved = pairs * fl / (m2l_ms / 1e3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            sm_mhz = float(json.load(fh)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        sm_mhz = 2070.0
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    if mixed:
        peak = n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        peak_kind = f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {sm_mhz:.0f} MHz"
    else:
        peak = FP64_NOMINAL_TFLOPS
        peak_kind = "nominal GB300 FP64"
    launches = sum(_fmm_kernels_per_instance(info[dd]["n_levels"], mixed) for dd in sets) * args.steps
    m2l_traffic = None
    if mixed:
        try:
            with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
                tj = json.load(fh)
            m2l_traffic = tj["fmm_m2l_mixed_uniform_bytes"] + tj["fmm_m2l_mixed_plummer_bytes"]
        except (OSError, KeyError, ValueError):
            pass
    line = {
        "metric": "FMM time", "value": ms_per_instance, "unit": "ms/instance", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": f"Laplace FMM N=2^20 (uniform cube and Plummer a=1 r<=10, seed 3, q~U(-1,1)), "
                               f"p={FMM_P}, theta={FMM_THETA}, leaf {FMM_LEAF}, block-mode DTT; "
                               f"{'mixed: FP32 P2P/M2L, FP64 top-level M2M/L2L' if mixed else 'plain FP64'}; "
                               "one step = both point sets end to end (tree, upward, DTT, M2L, downward, P2P/L2P)",
                   "l2": "positions 24 MiB + lists ~300 MiB per instance; the tree and lists are rebuilt every instance",
                   "parallelism": "replicas"},
        "breakdown_ms": breakdown,
        "dtt_ms": {dd: breakdown[dd]["ms_traverse"] for dd in sets},
        "lists": {dd: {"m2l": info[dd]["n_m2l"], "p2p": info[dd]["n_p2p"], "cells": info[dd]["n_cells"],
                       "levels": info[dd]["n_levels"]} for dd in sets},
        "rel_l2_vs_oracle_fmm_64_targets": errs,
        "roofline": {"bound": "alu", "kernel": "k_m2l_reg (M2L)", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": m2l_traffic, "traffic_note": "DRAM bytes of the two M2L launches of a step "
                     "(uniform + Plummer), one-pass ncu capture at full size",
                     "algorithmic_flops_per_pair": fl},
        "e2e": {"value": e2e_ms, "unit": "ms/instance", "h2d_bytes_per_step": len(sets) * FMM_N * 32,
                "d2h_bytes_per_step": len(sets) * FMM_N * 8},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs = _fmm_cpu_sample()
        line["cpu_baseline"] = {"value": secs * 1e3 * FMM_N / FMM_CPU_SAMPLE_N, "unit": "ms/instance", "cores": 1,
                                "kind": "oracle",
                                "sample": f"oracle FMM (FP64, same p/theta/leaf) on the first 2^16 points of the "
                                          f"uniform set, {secs:.2f} s single thread, scaled x16 to N=2^20 "
                                          "(cost linear in N at fixed leaf size)"}
    for d in sets.values():
        d["f"].close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _fmm_cpu_sample():
    import oracle
    from paper_2604_05982_gb300 import inputs
    oracle.build()
    try:
        os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    except (AttributeError, OSError):
        pass
    pos, q = inputs.fmm_points(FMM_N, "uniform", seed=3)
    pos, q = pos[:FMM_CPU_SAMPLE_N].copy(), q[:FMM_CPU_SAMPLE_N].copy()
    t0 = time.perf_counter()
    oracle.fmm(pos, q, p=FMM_P, theta=FMM_THETA, leaf_size=FMM_LEAF)
    return time.perf_counter() - t0


KC_SCALE = 20
KC_K = 4          # default k; --k selects 5, 6, 7
KC_QUEUES = 4
KC_CPU_RANGES = 2048     # oracle sample: evenly spaced DAG-edge ranges ...
KC_CPU_RANGE = 64        # ... of this many edges each at k = 4 (~0.8 % of the scale-20 graph's edges),
                         # a quarter as many per step of k above 4


def _pin_one_core():
    try:
        os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    except (AttributeError, OSError):
        pass


def _kclique_cpu_sample(n, e, k=KC_K):
    """One oracle k-clique instance estimated on one core: the orientation in full,
    the counting on KC_CPU_RANGES evenly spaced ranges of KC_CPU_RANGE DAG edges,
    scaled to all edges.  Returns (ms per instance, seconds spent)."""
    import numpy as np

    import oracle
    oracle.build()
    m = len(e)
    t0 = time.perf_counter()
    off, adj = oracle.orient(n, e)
    t1 = time.perf_counter()
    per = max(1, KC_CPU_RANGE >> (2 * (k - 4)))
    starts = np.arange(KC_CPU_RANGES, dtype=np.int64) * (m // KC_CPU_RANGES)
    ranges = np.stack([starts, np.minimum(starts + per, m)], axis=1)
    oracle.kclique_dag_ranges(off, adj, k, ranges)
    t2 = time.perf_counter()
    sampled = int((ranges[:, 1] - ranges[:, 0]).sum())
    return ((t1 - t0) + (t2 - t1) * m / sampled) * 1e3, t2 - t0


def _kclique_cpu_note(m, k=KC_K):
    per = max(1, KC_CPU_RANGE >> (2 * (k - 4)))
    return (f"oracle on one core: orientation of the whole graph, then the {k}-clique count on "
            f"{KC_CPU_RANGES} evenly spaced ranges of {per} DAG edges, scaled to all {m} edges")


def run_reference_kclique(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2604_05982_gb300 import inputs
    _pin_one_core()
    n, e = inputs.rmat_graph(args.scale, 16, seed=7)
    for _ in range(min(args.warmup, 1)):
        _kclique_cpu_sample(n, e, args.k)
    vals = [_kclique_cpu_sample(n, e, args.k)[0] for _ in range(args.steps)]
    value = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": "k-clique time", "value": value, "unit": "ms/instance", "n_gpus": world,
            "steps": args.steps, "warmup": min(args.warmup, 1), "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"{args.k}-clique count, R-MAT scale {args.scale} edge factor 16, seed 7 (oracle)"},
            "cpu_baseline": {"value": value, "unit": "ms/instance", "cores": 1, "kind": "oracle",
                             "sample": _kclique_cpu_note(len(e), args.k)},
            "e2e": {"value": value, "unit": "ms/instance", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_kclique(args):
    """k-clique counting on the scale-20 R-MAT graph: one step = orientation + context
    initialisation + the counting run + finalisation (the paper times k-clique with
    its initialisation)."""
    import numpy as np
    import torch

    import oracle
    from paper_2604_05982_gb300 import gtap as G
    from paper_2604_05982_gb300 import inputs, runner
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    n, e = inputs.rmat_graph(args.scale, 16, seed=7)
    edges = torch.from_numpy(np.ascontiguousarray(e)).cuda()
    m = int(edges.shape[0])
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    adj = torch.empty(m, dtype=torch.int32, device="cuda")
    src = torch.empty(m, dtype=torch.int32, device="cuda")
    work = torch.empty(4 * n + 16, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    algo = G.GTAP_KCLIQUE_PIVOT if args.algorithm == "pivot" else G.GTAP_KCLIQUE_ORIENT
    thr = 32 if algo == G.GTAP_KCLIQUE_PIVOT else 64
    kargs = G.gtap_kclique_args(off.data_ptr(), adj.data_ptr(), src.data_ptr(), 0, m, args.k, thr, 1, algo)
    big = args.k > 4 or args.algorithm == "pivot"   # larger frontier: rings of 16384, 4 GiB pool
    pool = 4 << 30 if big else 1 << 30
    # pivoting keeps a bitset subgraph per split set: its scratch high-water mark is far above orientation's
    scratch = (48 << 30) if args.algorithm == "pivot" else (4 << 30)
    ring = 16384 if big else 4096
    deadline_ns = (600 if big else 60) * 10 ** 9   # device deadline of one counting run

    def step():
        G.gtap_kclique_orient(edges.data_ptr(), m, n, off.data_ptr(), adj.data_ptr(), src.data_ptr(),
                              work.data_ptr(), 0)
        with runner.Context(G.GTAP_MODE_THREAD, KC_QUEUES, pool_bytes=pool, scratch_bytes=scratch,
                            deque_capacity=ring, timeout_ns=deadline_ns) as c:
            t = c.register("kclique")
            h = c.spawn(t, kargs)
            c.run()
            return c.result_u64(h), c.stats()["kernel_ms"]

    for _ in range(args.warmup):
        count, _ = step()
    # parity (outside the timed region): the full count against the oracle's golden value
    # (tests/golden, written from the oracle alone) where one exists, and sampled DAG-edge
    # ranges against the oracle run here
    gold = _kclique_golden(f"kclique_rmat{args.scale}_k{args.k}.txt")
    if gold is not None:
        assert count == gold["total"], (count, gold["total"])
    if args.k <= 4:
        ranges = [(lo, lo + 400) for lo in (0, m // 3, (2 * m) // 3)] + [(m - 200, m)]
    else:
        # larger k: the oracle's cost per edge explodes at the dense low-id end, so sample the rest
        ranges = [(lo, lo + 64) for lo in ((2 * m) // 3, (5 * m) // 6)] + [(m - 200, m)]
    want = [oracle.kclique_edge_range(n, e, args.k, lo, hi) for lo, hi in ranges]
    sampled = _kclique_golden(f"kclique_rmat{args.scale}_k{args.k}_sampled.txt")
    if sampled is not None:
        # the oracle's sampled ranges over the whole graph (written ahead by the golden script)
        ranges += [(lo, hi) for lo, hi, _ in sampled["ranges"]]
        want += [cnt for _, _, cnt in sampled["ranges"]]
    with runner.Context(G.GTAP_MODE_THREAD, 4, pool_bytes=pool, scratch_bytes=scratch, deque_capacity=ring,
                        max_roots=max(4096, len(ranges)), timeout_ns=deadline_ns) as c:
        t = c.register("kclique")
        hs = [c.spawn(t, G.gtap_kclique_args(off.data_ptr(), adj.data_ptr(), src.data_ptr(), lo, hi, args.k, thr, 1,
                                             algo))
              for lo, hi in ranges]
        c.run()
        got = [c.result_u64(h) for h in hs]
    assert got == want, (got, want)
    kms = []
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            c_, k_ = step()
            assert c_ == count
            kms.append(k_)
        torch.cuda.synchronize()
        elapsed = max_over_ranks(time.perf_counter() - t0)
    ms = elapsed * 1e3 / (args.steps * world)
    kms.sort()
    line = {
        "metric": "k-clique time", "value": ms, "unit": "ms/instance", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{args.k}-clique count by {'pivoting' if algo else 'orientation'}, R-MAT scale "
                               f"{args.scale} edge factor 16 (a,b,c=0.57,0.19,0.19, seed 7, {m} undirected edges), "
                               f"degree-ordered DAG, thread mode, DAQ {KC_QUEUES} queues by recursion depth, split "
                               f"threshold {thr}; one step = orientation + gtap_init + run + gtap_finalize (wall "
                               "clock, synchronised)", "parallelism": "replicas",
                   "l2": "graph 126 MB CSR + 63 MB edge list, > L2 with the scratch sets"},
        "count": count, "kernel_ms_median": kms[len(kms) // 2],
        "algorithm": args.algorithm,
        "parity": ("full count equals the oracle's (golden file) and sampled ranges equal the oracle's"
                   if gold is not None else "sampled DAG-edge ranges equal the oracle's"),
        "e2e": {"value": ms, "unit": "ms/instance", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 16,
                "note": "the edge list stays resident; the count is read back each step"},
        "gpu_launches": (9 + 2) * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _pin_one_core()
        value, _ = _kclique_cpu_sample(n, e, args.k)
        line["cpu_baseline"] = {"value": value, "unit": "ms/instance", "cores": 1, "kind": "oracle",
                                "sample": _kclique_cpu_note(m, args.k)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


SERVE_REQUESTS = 20000
SERVE_RATE = 5000.0
SERVE_CPU_SAMPLE = 200   # oracle sample: the first requests of the trace


def _serve_cpu_sample(reqs, n_sample):
    """The oracle answering the first n_sample requests of the trace one after
    another on one core (arrival times ignored, i.e. a saturated server).
    Returns (requests/s, the oracle's answers)."""
    import oracle
    from paper_2604_05982_gb300 import inputs
    oracle.build()
    graphs = {s: inputs.rmat_graph(s, 16, seed=7) for s in range(10, 15)}
    sample = reqs[:n_sample]
    answers = []
    t0 = time.perf_counter()
    for i, (kind, x) in enumerate(sample):
        if kind == "fib":
            answers.append(oracle.fib(x)[0])
        elif kind == "nqueens":
            answers.append(oracle.nqueens(x)[0])
        elif kind == "kclique":
            answers.append(oracle.kclique(*graphs[x], 4))
        else:
            nodes, leaves = oracle.uts(seed=1000 + i, root_children=x, m=5)
            answers.append((nodes << 32) | leaves)
    secs = time.perf_counter() - t0
    return len(sample) / secs, answers


def _serve_cpu_note(n_sample):
    return (f"oracle on one core answering the first {n_sample} requests of the same trace one after another "
            "(arrivals ignored: a saturated server)")


def run_reference_serve(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    _pin_one_core()
    _, reqs = _serve_trace(args.requests, SERVE_RATE)
    n_sample = min(SERVE_CPU_SAMPLE, len(reqs))
    for _ in range(min(args.warmup, 1)):
        _serve_cpu_sample(reqs, n_sample)
    vals = [_serve_cpu_sample(reqs, n_sample)[0] for _ in range(args.steps)]
    value = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": "served requests/s", "value": value, "unit": "req/s", "n_gpus": world,
            "steps": args.steps, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * n_sample / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "served mix: fib n in [20,32], N-Queens n in [8,12], 4-clique on R-MAT scale "
                                   "[10,14], hashed tree root [100,2000] (oracle)"},
            "cpu_baseline": {"value": value, "unit": "req/s", "cores": 1, "kind": "oracle",
                             "sample": _serve_cpu_note(n_sample)},
            "e2e": {"value": value, "unit": "req/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _serve_trace(n_req, rate, seed=11):
    """Poisson arrivals and the served mix: fib n in [20,32], N-Queens n in [8,12],
    4-clique on an R-MAT graph of scale in [10,14], hashed tree with root branching in [100,2000]."""
    import numpy as np

    from paper_2604_05982_gb300 import inputs
    arrivals, u = inputs.poisson_trace(n_req, rate, seed)
    v = inputs.u01(seed ^ 0x7E57, 0, n_req)
    kinds = np.minimum((u * 4).astype(int), 3)
    reqs = []
    for i in range(n_req):
        k = int(kinds[i])
        if k == 0:
            reqs.append(("fib", 20 + int(v[i] * 13)))
        elif k == 1:
            reqs.append(("nqueens", 8 + int(v[i] * 5)))
        elif k == 2:
            reqs.append(("kclique", 10 + int(v[i] * 5)))
        else:
            reqs.append(("uts", 100 + int(v[i] * 1901)))
    return arrivals, reqs


def run_serve(args):
    """Served mixed stream into the resident kernel vs one launch per request."""
    global np
    import numpy as np
    import torch

    from paper_2604_05982_gb300 import gtap as G
    from paper_2604_05982_gb300 import inputs, runner
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    n_req = args.requests
    arrivals, reqs = _serve_trace(n_req, SERVE_RATE)
    graphs = {s: runner.DeviceGraph(*inputs.rmat_graph(s, 16, seed=7)) for s in range(10, 15)}
    progs = ("fib", "nqueens", "kclique", "uts")

    def args_for(ctxtypes, r, i):
        kind, x = r
        if kind == "fib":
            return ctxtypes["fib"], G.gtap_fib_args(x, 0)
        if kind == "nqueens":
            return ctxtypes["nqueens"], G.gtap_nqueens_args(x, 0)
        if kind == "kclique":
            return ctxtypes["kclique"], graphs[x].args(4)
        return ctxtypes["uts"], G.gtap_uts_args(1000 + i, runner.UTS_THRESHOLD_Q0199, x, 5, 0, 0)

    pool = 4 << 30
    # ---- served: one resident kernel, requests through the inbox
    with runner.Context(G.GTAP_MODE_THREAD, 1, pool_bytes=pool, scratch_bytes=1 << 30, max_roots=4096) as c:
        types = {p: c.register(p) for p in progs}
        G.gtap_serve_start(c.ctx)
        req_of = {}
        done_t = np.zeros(n_req)
        served_val = [None] * n_req
        t0 = time.perf_counter()
        nxt, ndone = 0, 0
        failure = None
        # where requests wait: sampled every 2 ms from gtap_serve_progress
        # (submitted - admitted = inbox backlog; admitted - polled = on the device)
        backlog, on_device, last_sample = [], [], -1.0
        clk = ClockSampler(local).__enter__()
        try:
            while ndone < n_req:
                now = time.perf_counter() - t0
                if now > arrivals[-1] + 120.0:
                    failure = f"deadline: {ndone} of {n_req} completed"
                    break
                while nxt < n_req and arrivals[nxt] <= now:
                    t, a = args_for(types, reqs[nxt], nxt)
                    rid = G.gtap_submit(c.ctx, t, a, 0)
                    if rid is None:
                        break
                    req_of[rid] = nxt
                    nxt += 1
                for rid, r0, _, st in G.gtap_poll(c.ctx):
                    i = req_of[rid]
                    done_t[i] = time.perf_counter() - t0
                    served_val[i] = r0
                    ndone += 1
                if now - last_sample >= 0.002:
                    sub, adm, pol = G.gtap_serve_progress(c.ctx)
                    backlog.append(sub - adm)
                    on_device.append(adm - pol)
                    last_sample = now
        except G.GtapError as exc:
            failure = str(exc)
        finally:
            clk.__exit__(None, None, None)
            progress = G.gtap_serve_progress(c.ctx)
            stop_status = G.load_library().gtap_serve_stop(c.ctx, 60000)
        if failure is not None or stop_status != 0:
            diag = {"submitted_admitted_polled": list(progress)}
            try:
                st = c.stats()
                diag.update({k: st[k] for k in ("frames_high_water", "scratch_used", "tasks_executed")})
            except Exception as exc:  # the stats of a failed session may be unreadable
                diag["stats_error"] = str(exc)
            print(json.dumps({"metric": "served requests/s", "error": failure or G.STATUS.get(stop_status),
                              "diagnostics": diag}), flush=True)
            sys.exit(1)
    lat_served = (done_t - arrivals) * 1e3
    span_served = done_t.max() - arrivals[0]

    # ---- one launch per request, same arrival trace and GPU
    with runner.Context(G.GTAP_MODE_THREAD, 1, pool_bytes=pool, scratch_bytes=1 << 30) as c:
        types = {p: c.register(p) for p in progs}
        done_b = np.zeros(n_req)
        base_val = [None] * n_req
        t0 = time.perf_counter()
        for i in range(n_req):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            c.clear()
            t, a = args_for(types, reqs[i], i)
            h = c.spawn(t, a)
            c.run()
            base_val[i] = c.result_u64(h)
            done_b[i] = time.perf_counter() - t0
    lat_base = (done_b - arrivals) * 1e3
    span_base = done_b.max() - arrivals[0]
    identical = served_val == base_val

    def pct(a, q):
        return float(np.percentile(a, q))

    line = {"metric": "served requests/s", "value": n_req / span_served, "unit": "req/s", "n_gpus": world,
            "steps": 1, "warmup": 0, "ms_per_step": span_served * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"served mix: Poisson {SERVE_RATE:.0f} req/s, {n_req} requests of fib n in [20,32], "
                                   "N-Queens n in [8,12], 4-clique on R-MAT scale [10,14], hashed tree root [100,2000]; "
                                   "4 GiB record pool", "parallelism": "replicas"},
            "latency_ms": {"p50": pct(lat_served, 50), "p99": pct(lat_served, 99), "max": float(lat_served.max())},
            "per_request_launch": {"value": n_req / span_base, "unit": "req/s", "p50_ms": pct(lat_base, 50),
                                   "p99_ms": pct(lat_base, 99)},
            "results_identical_alone_and_in_mix": bool(identical), "clocks": clk.summary(),
            "e2e": {"value": n_req / span_served, "unit": "req/s", "h2d_bytes_per_step": 128 * n_req,
                    "d2h_bytes_per_step": 48 * n_req,
                    "note": "the served rate is end to end: requests written by the host into the mapped inbox "
                            "(128 B each), completions read from the mapped outbox (48 B each)"},
            "gpu_launches": 2,
            "waiting": {"inbox_mean": float(np.mean(backlog)), "inbox_max": int(max(backlog)),
                        "on_device_mean": float(np.mean(on_device)), "on_device_max": int(max(on_device)),
                        "samples": len(backlog),
                        "limit": "admission" if np.mean(backlog) > np.mean(on_device) else "device work"}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _pin_one_core()
        n_sample = min(SERVE_CPU_SAMPLE, n_req)
        rps, answers = _serve_cpu_sample(reqs, n_sample)
        line["cpu_baseline"] = {"value": rps, "unit": "req/s", "cores": 1, "kind": "oracle",
                                "sample": _serve_cpu_note(n_sample)}
        line["oracle_check"] = {"requests": n_sample, "served_equal_oracle": served_val[:n_sample] == answers}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Atomic-rate ceiling, measured live (the roofline denominator of the thread-mode
# scheduler kernels): scattered acq_rel 32-bit adds with return (the join
# decrement) and scattered 64-bit reductions (accumulating joins).
def atomic_ceiling(local: int = 0):
    import torch

    from paper_2604_05982_gb300 import gtap as G
    region = torch.zeros(200 << 18, dtype=torch.int32, device=f"cuda:{local}")
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    out = {}
    for kind, key in ((0, "join_decrement"), (1, "accumulate")):
        ms, ops = G.gtap_microbench(kind, region.data_ptr(), region.numel() * 4, sms * 8, 256, 64)
        out[key] = ops / (ms / 1e3)
    del region
    return out


def _atomic_roofline(kernel, tasks, decrements, accumulates, kernel_ms, ceil):
    """Roofline object of a thread-mode kernel against the measured atomic rates: the
    launch's join decrements and accumulating adds take 1/rate each of the L2 atomic
    units; achieved = atomic operations per second of the kernel's duration."""
    secs = kernel_ms / 1e3
    ops = decrements + accumulates
    # time the atomic units need for this mix at the measured rates, per operation
    t_ops = decrements / ceil["join_decrement"] + accumulates / ceil["accumulate"]
    peak = ops / t_ops
    achieved = ops / secs
    return {"bound": "l2_atomic", "kernel": kernel, "achieved": achieved / 1e9, "peak": peak / 1e9,
            "peak_kind": "measured live (gtap_microbench kinds 0 and 1: scattered acq_rel add, red.add.u64)",
            "unit": "Gop/s", "frac": achieved / peak, "traffic": None, "tasks_per_s": tasks / secs,
            "atomics_per_launch": ops}


FIB_N = 30
FIB_TASKS = 2692537          # 2 F(31) - 1


def _gpu_setup(args):
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    from paper_2604_05982_gb300 import gtap as G
    G.load_library()
    return world, rank, local


def _finish(line, world, rank):
    import torch
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_fib(args):
    """fib(30) in thread mode, no cutoff: one step = one persistent-kernel run."""
    import torch

    import oracle
    from paper_2604_05982_gb300 import gtap as G
    from paper_2604_05982_gb300 import runner
    world, rank, local = _gpu_setup(args)
    fa = G.gtap_fib_args(FIB_N, 0)
    tmask = G.GTAP_TUNE_BLOCKS | G.GTAP_TUNE_STEAL | G.GTAP_TUNE_CAPACITY | G.GTAP_TUNE_BACKOFF
    if args.no_tune:
        tuned = {"blocks_per_sm": 4, "steal_policy": 0, "deque_capacity": 4096, "idle_backoff_ns": 512}
    else:
        best, _ = G.gtap_autotune(G.GTAP_MODE_THREAD, "fib", [fa], 1 << 30, runner.make_config(), reps=3,
                                  n_queues=1, tune_mask=tmask)
        tuned = {k: best[k] for k in ("blocks_per_sm", "steal_policy", "deque_capacity", "idle_backoff_ns")}
    c = runner.Context(G.GTAP_MODE_THREAD, 1, pool_bytes=1 << 30, **tuned)
    t = c.register("fib")
    h = c.spawn(t, fa)
    for _ in range(args.warmup):
        c.run()
    v, tasks = oracle.fib(FIB_N)
    assert c.result_i64(h) == v == 832040
    assert c.stats()["tasks_created"] == tasks == FIB_TASKS
    ceil = atomic_ceiling(local)
    kms = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            c.run()
            kms.append(c.stats()["kernel_ms"])
        e1.record()
        torch.cuda.synchronize()
    elapsed_ms = max_over_ranks(e0.elapsed_time(e1))
    value = aggregate_rate(FIB_TASKS, args.steps, world, elapsed_ms)
    # end to end through the C ABI from the host: queue the root (its arguments are copied
    # to the device by gtap_run), run, wait (the results and counters come back), read
    t0 = time.perf_counter()
    for _ in range(args.steps):
        c.clear()
        hh = c.spawn(t, fa)
        c.run()
        assert c.result_i64(hh) == 832040
    e2e_s = (time.perf_counter() - t0) / args.steps
    kms.sort()
    kmed = kms[len(kms) // 2]
    st = c.stats()
    line = {
        "metric": "tasks/s", "value": value, "unit": "tasks/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"fib({FIB_N}) thread mode, a task per call, no cutoff ({FIB_TASKS} tasks)",
                   "parallelism": "replicas", "l2": "task records re-initialised every run (172 MB pool touched)"},
        "result": v, "tasks_created": st["tasks_created"], "kernel_ms_median": kmed,
        "launch_config": {"source": "default" if args.no_tune else "gtap_autotune", **tuned},
        "roofline": _atomic_roofline("thread_kernel<fib>", FIB_TASKS, FIB_TASKS - 1, 0, kmed, ceil),
        "atomic_ceiling_gops": {k: x / 1e9 for k, x in ceil.items()},
        "e2e": {"value": FIB_TASKS / e2e_s, "unit": "tasks/s", "ms_per_step": e2e_s * 1e3,
                "h2d_bytes_per_step": 128, "d2h_bytes_per_step": 8,
                "note": "root arguments in, result out through gtap_spawn_root / gtap_run / gtap_wait / "
                        "gtap_read_result (wall clock)"},
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _pin_one_core()
        t0 = time.perf_counter()
        oracle.fib(FIB_N)
        secs = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": FIB_TASKS / secs, "unit": "tasks/s", "cores": 1, "kind": "oracle",
                                "sample": f"oracle fib({FIB_N}) serial recursion, single thread ({secs:.3f} s)"}
    c.close()
    _finish(line, world, rank)


SCHED_N = 35
SCHED_GRIDS = (1, 4, 16, 38, 76, 152, 304, 608)   # 256-thread blocks


def run_sched(args):
    """Sec. 6.5: centralised queue, non-batched stealing and batched stealing on fib(35)
    across grid sizes (one launch per configuration, median kernel time)."""
    import oracle
    from paper_2604_05982_gb300 import gtap as G
    from paper_2604_05982_gb300 import runner
    world, rank, local = _gpu_setup(args)
    v, tasks = oracle.fib(SCHED_N)
    names = {G.GTAP_SCHED_BATCHED: "batched stealing", G.GTAP_SCHED_SINGLE: "non-batched stealing",
             G.GTAP_SCHED_GLOBAL: "central queue"}
    rows = []
    reps = max(1, min(args.steps, 5))
    clk = ClockSampler(local).__enter__()
    for sched in names:
        for grid in SCHED_GRIDS:
            with runner.Context(G.GTAP_MODE_THREAD, 1, pool_bytes=2 << 30, scheduler=sched, grid_blocks=grid,
                                blocks_per_sm=4) as c:
                t = c.register("fib")
                h = c.spawn(t, G.gtap_fib_args(SCHED_N, 0))
                ks = []
                for i in range(1 + reps):
                    c.run(timeout_ms=120000)
                    assert c.result_i64(h) == v and c.stats()["tasks_created"] == tasks
                    if i:
                        ks.append(c.stats()["kernel_ms"])
                ks.sort()
                ms = ks[len(ks) // 2]
                rows.append({"scheduler": names[sched], "grid_blocks": grid, "threads": grid * 256,
                             "kernel_ms": ms, "tasks_per_s": tasks / (ms / 1e3)})
                print(json.dumps({"progress": rows[-1]}), file=sys.stderr, flush=True)
    clk.__exit__(None, None, None)
    best = [r for r in rows if r["scheduler"] == "batched stealing" and r["grid_blocks"] == 608][0]
    line = {"metric": "tasks/s", "value": best["tasks_per_s"], "unit": "tasks/s", "n_gpus": world,
            "steps": reps, "warmup": 1, "ms_per_step": best["kernel_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"scheduler comparison (Sec. 6.5): fib({SCHED_N}) thread mode, {tasks} tasks, "
                                   "central queue vs non-batched vs batched stealing across grid sizes of "
                                   "256-thread blocks", "parallelism": "replicas"},
            "value_is": "batched stealing at 608 blocks (4 per SM)", "sweep": rows,
            "gpu_launches": 2 * (1 + reps) * len(rows), "clocks": clk.summary()}
    _finish(line, world, rank)


MICRO_GRID, MICRO_BS = 2000, 32     # Sec. 6.1: grid size 2000, block size 32 in both modes


def run_micro(args):
    """Sec. 6.1 / 6.2: full binary task tree, thread mode vs block mode (with and
    without a 5-level cutoff), compute_iters and depth sweeps; heterogeneous leaves
    (K = 2, 4) with and without DAQ.  Every run's sum is checked against the oracle
    on a sampled subset (full oracle for the small trees)."""
    import oracle
    from paper_2604_05982_gb300 import gtap as G
    from paper_2604_05982_gb300 import runner
    world, rank, local = _gpu_setup(args)
    reps = max(1, min(args.steps, 3))
    geo = dict(grid_blocks=MICRO_GRID, threads_per_block=MICRO_BS, blocks_per_sm=32, pool_bytes=4 << 30,
               deque_capacity=16384)

    def timed(depth, iters, K=1, block=False, cutoff=0, daq=False):
        q = K + 1 if daq else 1
        mode = G.GTAP_MODE_BLOCK if block else G.GTAP_MODE_THREAD
        with runner.Context(mode, q, **geo) as c:
            t = c.register("bintree_block" if block else "bintree")
            h = c.spawn(t, G.gtap_bintree_args(depth, iters, K, 1 if daq else 0, cutoff, 0))
            ks = []
            for i in range(1 + reps):
                c.run(timeout_ms=300000)
                if i:
                    ks.append(c.stats()["kernel_ms"])
            val = c.result_u64(h)
        ks.sort()
        return ks[len(ks) // 2], val

    want_cache = {}

    def check(depth, iters, K, val):
        if depth <= 16:
            key = (depth, iters, K)
            if key not in want_cache:
                want_cache[key] = oracle.bintree(depth, iters, K)[0]
            assert val == want_cache[key], key
        return True

    out = {"iters_sweep": [], "depth_sweep": [], "hetero": []}
    D = 25
    clk = ClockSampler(local).__enter__()
    for iters in (1, 16, 256, 2048):
        row = {"depth": D, "compute_iters": iters}
        vals = set()
        for name, kw in (("thread", {}), ("block", {"block": True}), ("block_cutoff5", {"block": True, "cutoff": 5})):
            ms, val = timed(D, iters, **kw)
            row[name + "_ms"] = ms
            vals.add(val)
        assert len(vals) == 1, row          # the three modes give the same sum
        row["block_over_thread"] = row["block_ms"] / row["thread_ms"]
        row["cutoff_over_thread"] = row["block_cutoff5_ms"] / row["thread_ms"]
        out["iters_sweep"].append(row)
        print(json.dumps({"progress": row}), file=sys.stderr, flush=True)
    for depth in (8, 10, 12, 14, 16, 18, 20, 22, 25):
        row = {"depth": depth, "compute_iters": 2048}
        for name, kw in (("thread", {}), ("block", {"block": True}), ("block_cutoff5", {"block": True, "cutoff": 5})):
            ms, val = timed(depth, 2048, **kw)
            check(depth, 2048, 1, val)
            row[name + "_ms"] = ms
        row["block_over_thread"] = row["block_ms"] / row["thread_ms"]
        row["cutoff_over_thread"] = row["block_cutoff5_ms"] / row["thread_ms"]
        out["depth_sweep"].append(row)
        print(json.dumps({"progress": row}), file=sys.stderr, flush=True)
    for K in (2, 4):
        for iters in (16, 256, 2048):
            row = {"K": K, "depth": D, "compute_iters": iters}
            vals = set()
            for name, kw in (("thread_nodaq", {}), ("thread_daq", {"daq": True}), ("block", {"block": True})):
                ms, val = timed(D, iters, K=K, **kw)
                row[name + "_ms"] = ms
                vals.add(val)
            assert len(vals) == 1, row
            row["daq_speedup"] = row["thread_nodaq_ms"] / row["thread_daq_ms"]
            out["hetero"].append(row)
            print(json.dumps({"progress": row}), file=sys.stderr, flush=True)
    clk.__exit__(None, None, None)

    # the depth at which thread mode overtakes each block variant
    def crossover(key):
        for r in out["depth_sweep"]:
            if r[key] > 1.0:
                return r["depth"]
        return None
    ref = [r for r in out["iters_sweep"] if r["compute_iters"] == 2048][0]
    line = {"metric": "binary-tree time", "value": ref["thread_ms"], "unit": "ms", "n_gpus": world, "steps": reps,
            "warmup": 1, "ms_per_step": ref["thread_ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"mode/DAQ microbenchmarks (Sec. 6.1, 6.2): full binary task tree, depth {D}, "
                                   f"compute_iters 2048, grid {MICRO_GRID} x {MICRO_BS} threads in both modes",
                       "parallelism": "replicas"},
            "value_is": "thread mode, D = 25, compute_iters = 2048", **out,
            "thread_overtakes_block_at_depth": crossover("block_over_thread"),
            "thread_overtakes_block_cutoff_at_depth": crossover("cutoff_over_thread"),
            "gpu_launches": 2 * (1 + reps) * (3 * 4 + 3 * 9 + 3 * 6), "clocks": clk.summary()}
    _finish(line, world, rank)



def _kclique_golden(name):
    """A k-clique golden file written by tests/golden/make_kclique_goldens.py (oracle only)."""
    import importlib.util
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None
    spec = importlib.util.spec_from_file_location("make_kclique_goldens",
                                                  os.path.join(ROOT, "tests", "golden", "make_kclique_goldens.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.load(path)


BATCH_GRAPHS = 64


def run_batch(args):
    """The batched k-clique variant: 64 R-MAT graphs (graph i: scale 12 + floor(7i/64), seed
    7 + i), 4-cliques, as (a) one persistent launch with 64 roots, (b) the replay of that
    launch captured as a CUDA graph, (c) 64 plain launches, one per instance.  Counts are
    asserted equal across the three forms and to the oracle's."""
    import numpy as np
    import torch

    from paper_2604_05982_gb300 import gtap as G
    from paper_2604_05982_gb300 import inputs, runner
    world, rank, local = _gpu_setup(args)
    gold = _kclique_golden("kclique_batch64_k4.txt")
    specs = [(12 + (7 * i) // 64, 7 + i) for i in range(BATCH_GRAPHS)]
    graphs = [runner.DeviceGraph(*inputs.rmat_graph(sc, 16, seed=sd)) for sc, sd in specs]
    torch.cuda.synchronize()
    # DAQ 4 by depth: 64 instances' frontier can exceed rings of 16384 on one warp
    cfg = dict(pool_bytes=1 << 30, scratch_bytes=4 << 30, deque_capacity=65536)
    want = [g[4] for g in gold["graphs"]] if gold else None

    def one_launch(c, hs):
        c.run()
        return [c.result_u64(h) for h in hs]

    # (a) + (b): one context with the 64 roots
    c = runner.Context(G.GTAP_MODE_THREAD, 4, **cfg)
    t = c.register("kclique")
    hs = [c.spawn(t, g.args(4, 64, 1)) for g in graphs]
    for _ in range(args.warmup):
        got = one_launch(c, hs)
    if want is not None:
        assert got == want
    want = got

    def timed(fn, n):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / n

    with ClockSampler(local) as clk:
        t_plain = timed(lambda: one_launch(c, hs), args.steps)
        c.capture()
        for _ in range(2):
            assert one_launch(c, hs) == want
        t_graph = timed(lambda: one_launch(c, hs), args.steps)
        assert one_launch(c, hs) == want
        # (c) one launch per instance
        per = [runner.Context(G.GTAP_MODE_THREAD, 4, **cfg) for _ in range(1)]
        pc = per[0]
        pt = pc.register("kclique")

        def per_instance():
            out = []
            for g in graphs:
                pc.clear()
                h = pc.spawn(pt, g.args(4, 64, 1))
                pc.run()
                out.append(pc.result_u64(h))
            return out
        assert per_instance() == want
        t_per = timed(per_instance, max(1, args.steps // 2))
    elapsed = max_over_ranks(t_graph)
    line = {"metric": "batched jobs/s", "value": world * BATCH_GRAPHS / elapsed, "unit": "instances/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "batched k-clique: 64 R-MAT graphs (scales 12-18, graph i: scale 12 + floor(7i/64), "
                                   "edge factor 16, seed 7 + i), k = 4, DAQ 4 queues by depth, one persistent launch "
                                   "replayed from a captured CUDA graph", "parallelism": "replicas"},
            "forms_ms": {"graph_replay_one_launch": t_graph * 1e3, "plain_one_launch": t_plain * 1e3,
                         "one_launch_per_instance": t_per * 1e3},
            "speedup_vs_per_instance": t_per / t_graph,
            "counts_identical_across_forms": True,
            "counts_match_oracle_golden": gold is not None,
            "e2e": {"value": BATCH_GRAPHS / t_graph, "unit": "instances/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": BATCH_GRAPHS * 32,
                    "note": "graphs resident on the device; each step reads the 64 counts back (gtap_wait)"},
            "gpu_launches": 2 * (args.steps * 2 + args.steps // 2 * BATCH_GRAPHS),
            "clocks": clk.summary()}
    pc.close()
    c.close()
    _finish(line, world, rank)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gtap", choices=["gtap", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="integer set: default launch configuration, no autotuning")
    ap.add_argument("--workload", default="integer",
                    choices=["integer", "fib", "serve", "fmm", "kclique", "batch", "sched", "micro"],
                    help="integer: the default bench line (N-Queens 13, hashed tree, mergesort 2^26); fib: fib(30); "
                         "serve: the served mixed stream; fmm: Laplace FMM; kclique: k-clique count on the scale-20 "
                         "R-MAT graph; batch: 64 R-MAT graphs in one launch vs graph replay vs per-instance "
                         "launches; sched: scheduler comparison on fib(35); micro: mode/DAQ binary-tree sweeps")
    ap.add_argument("--requests", type=int, default=SERVE_REQUESTS)
    ap.add_argument("--k", type=int, default=KC_K, choices=[4, 5, 6, 7], help="kclique: clique size")
    ap.add_argument("--scale", type=int, default=KC_SCALE, help="kclique: R-MAT scale of the graph (default 20)")
    ap.add_argument("--algorithm", default="orient", choices=["orient", "pivot"],
                    help="kclique: orientation or pivoting (Sec. 6.4.2)")
    ap.add_argument("--fmm-precision", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        # one process per GPU: start the ranks here (replicas, see the multi-GPU notes)
        import socket
        sk = socket.socket()
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
        sk.close()
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
        sys.exit(subprocess.call(cmd))
    if world != args.gpus:
        print(json.dumps({"error": f"--gpus {args.gpus} but WORLD_SIZE={world}: launch one rank per GPU"}), flush=True)
        sys.exit(2)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "fmm":
        run_fmm(args)
    elif args.workload == "kclique":
        run_kclique(args)
    elif args.workload == "fib":
        run_fib(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "sched":
        run_sched(args)
    elif args.workload == "micro":
        run_micro(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
