"""Write the k-clique golden files from the CPU oracle alone.

Every value written here comes from ``oracle`` (the serial elision of the
k-clique program, Sec. 6.4.2) on graphs from the seeded generator in
``paper_2604_05982_gb300.inputs``; nothing is taken from the GPU path.

Files (one ``key value`` or ``range lo hi count`` record per line):

* ``kclique_rmat20_k{K}.txt``: the R-MAT graph of scale 20, edge factor 16,
  (a, b, c) = (0.57, 0.19, 0.19), seed 7, oriented by (degree, id).  The DAG
  edges [0, m) are cut into 64 contiguous ranges of (nearly) equal length; the
  file holds the count of each range and their sum, the whole graph's count.
* ``kclique_rmat20_k{K}_sampled.txt``: for k whose whole-graph count is out of
  the oracle's reach, ranges of a few DAG edges at evenly spaced starts.
* ``kclique_batch64_k4.txt``: the 64-graph batch, graph i of scale
  12 + floor(7 i / 64) and seed 7 + i, one 4-clique count per graph.

The oracle itself is single-threaded; this script only spreads independent
sub-ranges (or graphs) over worker processes and adds the integer results.

    python tests/golden/make_kclique_goldens.py rmat20 --k 4 --workers 8
    python tests/golden/make_kclique_goldens.py batch64 --workers 8
    python tests/golden/make_kclique_goldens.py rmat20 --k 6 --sample 256 --width 4 --workers 8
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_RANGES = 64          # golden ranges per graph
SUB_PER_RANGE = 64     # work items per golden range (load balance: low vertex ids carry most of the work)

_G = {}


def batch64_graph(i: int):
    """(scale, seed) of graph i of the 64-graph batch."""
    return 12 + (7 * i) // 64, 7 + i


def golden_ranges(m: int, n_ranges: int = N_RANGES):
    """Contiguous DAG-edge ranges [lo, hi) that partition [0, m)."""
    return [(i * m // n_ranges, (i + 1) * m // n_ranges) for i in range(n_ranges)]


def _init_rmat(scale: int, seed: int):
    import oracle
    from paper_2604_05982_gb300 import inputs
    n, e = inputs.rmat_graph(scale, 16, seed=seed)
    off, adj = oracle.orient(n, e)
    _G["off"], _G["adj"] = off, adj


def _count_range(job):
    import oracle
    idx, lo, hi, k = job
    t0 = time.perf_counter()
    c = oracle.kclique_dag_ranges(_G["off"], _G["adj"], k, [(lo, hi)]) if hi > lo else 0
    return idx, c, time.perf_counter() - t0


def _count_graph(job):
    import oracle
    from paper_2604_05982_gb300 import inputs
    i, k = job
    scale, seed = batch64_graph(i)
    n, e = inputs.rmat_graph(scale, 16, seed=seed)
    t0 = time.perf_counter()
    c = oracle.kclique(n, e, k)
    return i, scale, seed, len(e), c, time.perf_counter() - t0


def make_rmat20(k: int, workers: int, out: str):
    from paper_2604_05982_gb300 import inputs
    n, e = inputs.rmat_graph(20, 16, seed=7)
    m = len(e)
    ranges = golden_ranges(m)
    jobs = []
    for r, (lo, hi) in enumerate(ranges):
        for s in range(SUB_PER_RANGE):
            a = lo + s * (hi - lo) // SUB_PER_RANGE
            b = lo + (s + 1) * (hi - lo) // SUB_PER_RANGE
            jobs.append((r, a, b, k))
    # the expensive sub-ranges (low vertex ids) first, so the pool ends together
    ctx = mp.get_context("spawn")
    sums = [0] * len(ranges)
    t0 = time.perf_counter()
    cpu = 0.0
    with ctx.Pool(workers, initializer=_init_rmat, initargs=(20, 7)) as pool:
        for done, (r, c, secs) in enumerate(pool.imap_unordered(_count_range, jobs, chunksize=1)):
            sums[r] += c
            cpu += secs
            if done % 256 == 0:
                print(f"  {done}/{len(jobs)} sub-ranges, {time.perf_counter() - t0:.0f} s", flush=True)
    total = sum(sums)
    with open(out, "w") as f:
        f.write(f"# {k}-clique counts of the R-MAT graph scale 20, edge factor 16, a/b/c 0.57/0.19/0.19, seed 7\n")
        f.write("# (duplicates and self loops removed), DAG oriented by (degree, id) (Sec. 6.4.2).\n")
        f.write(f"# Written by tests/golden/make_kclique_goldens.py from the CPU oracle only "
                f"({cpu:.0f} s of oracle time).\n")
        f.write("# range lo hi: the count over DAG edges [lo, hi); the ranges partition [0, m).\n")
        f.write(f"n {n}\nm {m}\nk {k}\ntotal {total}\n")
        for (lo, hi), c in zip(ranges, sums):
            f.write(f"range {lo} {hi} {c}\n")
    print(f"total {total} ({time.perf_counter() - t0:.0f} s wall)")


def sampled_ranges(m: int, n_ranges: int, width: int):
    """n_ranges ranges of `width` DAG edges at evenly spaced starts over [0, m)."""
    return [(i * (m // n_ranges), min(m, i * (m // n_ranges) + width)) for i in range(n_ranges)]


def make_rmat20_sampled(k: int, workers: int, n_ranges: int, width: int, out: str):
    from paper_2604_05982_gb300 import inputs
    n, e = inputs.rmat_graph(20, 16, seed=7)
    m = len(e)
    ranges = sampled_ranges(m, n_ranges, width)
    ctx = mp.get_context("spawn")
    counts = [0] * len(ranges)
    t0 = time.perf_counter()
    cpu = 0.0
    with ctx.Pool(workers, initializer=_init_rmat, initargs=(20, 7)) as pool:
        jobs = [(r, lo, hi, k) for r, (lo, hi) in enumerate(ranges)]
        for done, (r, c, secs) in enumerate(pool.imap_unordered(_count_range, jobs, chunksize=1)):
            counts[r] = c
            cpu += secs
            if done % 32 == 0:
                print(f"  {done}/{len(jobs)} ranges, {time.perf_counter() - t0:.0f} s", flush=True)
    with open(out, "w") as f:
        f.write(f"# {k}-clique counts of sampled DAG-edge ranges of the R-MAT graph scale 20, edge factor 16,\n")
        f.write("# a/b/c 0.57/0.19/0.19, seed 7, oriented by (degree, id) (Sec. 6.4.2): the whole graph's count\n")
        f.write(f"# is out of the oracle's reach at this k, so {n_ranges} ranges of {width} edges at evenly spaced\n")
        f.write(f"# starts.  Written by tests/golden/make_kclique_goldens.py from the CPU oracle only "
                f"({cpu:.0f} s of oracle time).\n")
        f.write(f"n {n}\nm {m}\nk {k}\n")
        for (lo, hi), c in zip(ranges, counts):
            f.write(f"range {lo} {hi} {c}\n")
    print(f"done ({time.perf_counter() - t0:.0f} s wall)")


def make_batch64(k: int, workers: int, out: str):
    ctx = mp.get_context("spawn")
    rows = [None] * 64
    t0 = time.perf_counter()
    # the largest graphs first
    with ctx.Pool(workers) as pool:
        for i, scale, seed, m, c, secs in pool.imap_unordered(_count_graph, [(i, k) for i in reversed(range(64))]):
            rows[i] = (scale, seed, m, c)
            print(f"  graph {i} scale {scale}: {c} ({secs:.0f} s)", flush=True)
    with open(out, "w") as f:
        f.write(f"# {k}-clique counts of the 64-graph batch: graph i is R-MAT of scale 12 + floor(7 i / 64),\n")
        f.write("# edge factor 16, a/b/c 0.57/0.19/0.19, seed 7 + i, oriented by (degree, id) (Sec. 6.4.2).\n")
        f.write("# Written by tests/golden/make_kclique_goldens.py from the CPU oracle only.\n")
        f.write("# graph i scale seed m count\n")
        f.write(f"k {k}\n")
        for i, (scale, seed, m, c) in enumerate(rows):
            f.write(f"graph {i} {scale} {seed} {m} {c}\n")
    print(f"done ({time.perf_counter() - t0:.0f} s wall)")


def load(path: str) -> dict:
    """Parse a golden file into {'total': .., 'ranges': [(lo, hi, c)], 'graphs': [(i, scale, seed, m, c)], ...}."""
    out = {"ranges": [], "graphs": []}
    with open(path) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "range":
                out["ranges"].append(tuple(int(x) for x in t[1:4]))
            elif t[0] == "graph":
                out["graphs"].append(tuple(int(x) for x in t[1:6]))
            else:
                out[t[0]] = int(t[1])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["rmat20", "batch64"])
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--sample", type=int, default=0, help="rmat20: sampled ranges instead of the whole graph")
    ap.add_argument("--width", type=int, default=4, help="rmat20 --sample: DAG edges per range")
    a = ap.parse_args()
    if a.what == "rmat20" and a.sample:
        make_rmat20_sampled(a.k, a.workers, a.sample, a.width,
                            os.path.join(HERE, f"kclique_rmat20_k{a.k}_sampled.txt"))
    elif a.what == "rmat20":
        make_rmat20(a.k, a.workers, os.path.join(HERE, f"kclique_rmat20_k{a.k}.txt"))
    else:
        make_batch64(a.k, a.workers, os.path.join(HERE, f"kclique_batch64_k{a.k}.txt"))


if __name__ == "__main__":
    main()
