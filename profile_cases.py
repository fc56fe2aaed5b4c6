"""Single-workload runs for profiler captures (ncu): python profile_cases.py CASE ...

Each case runs one workload `--reps` times through the C ABI and prints the
kernel time of every run.  Used to capture one kernel of one workload with
ncu at a size that keeps the capture short.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["fib", "nqueens", "tree", "mergesort", "kclique", "fmm", "bintree"])
    ap.add_argument("--n", type=int, default=0, help="problem size (fib n, queens n, log2 keys, rmat scale)")
    ap.add_argument("--queues", type=int, default=1)
    ap.add_argument("--route", type=int, default=0)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--dist", default="uniform", help="fmm point set: uniform or plummer")
    ap.add_argument("--mixed", type=int, default=1, help="fmm: 1 mixed precision, 0 FP64")
    ap.add_argument("--sched", type=int, default=0, help="fib/tree: GTAP_SCHED_* scheduler variant")
    ap.add_argument("--iters", type=int, default=256, help="bintree: compute_iters")
    ap.add_argument("--K", type=int, default=1, help="bintree: leaf compute functions")
    ap.add_argument("--k", type=int, default=4, help="kclique: clique size")
    ap.add_argument("--block", type=int, default=0, help="bintree: 1 block mode")
    ap.add_argument("--grid", type=int, default=0, help="explicit grid size (0: the default)")
    ap.add_argument("--cutoff", type=int, default=0, help="fib / nqueens: sequential cutoff (0: none)")
    ap.add_argument("--sub", type=int, default=0, help="mergesort: log2 keys per independent sort (0: one sort)")
    args = ap.parse_args(argv)

    from paper_2604_05982_gb300 import gtap as G
    from paper_2604_05982_gb300 import inputs, runner
    geo = {"grid_blocks": args.grid} if args.grid else {}

    if args.case == "fib":
        for _ in range(args.reps):
            r = runner.fib(args.n or 30, n_queues=args.queues, route=args.route, cutoff=args.cutoff,
                           scheduler=args.sched, **geo)
            print("fib", r.values, r.stats["kernel_ms"])
    elif args.case == "nqueens":
        for _ in range(args.reps):
            r = runner.nqueens(args.n or 13, n_queues=args.queues, route=args.route, cutoff=args.cutoff, **geo)
            print("nqueens", r.values, r.stats["kernel_ms"])
    elif args.case == "tree":
        for _ in range(args.reps):
            r = runner.uts(42, n_queues=args.queues, route=args.route, scheduler=args.sched, **geo)
            print("tree", r.values, r.stats["kernel_ms"])
    elif args.case == "mergesort":
        import numpy as np
        import torch

        n = 1 << (args.n or 24)
        keys = inputs.keys_u32(n, seed=1)
        src = torch.from_numpy(keys.view(np.int32)).cuda()
        dst = torch.empty_like(src)
        tmp = torch.empty_like(src)
        torch.cuda.synchronize()
        sub = (1 << args.sub) if args.sub else n      # independent sorts of `sub` keys, one root each
        for _ in range(args.reps):
            with runner.Context(G.GTAP_MODE_BLOCK, 1, pool_bytes=256 << 20, max_roots=max(4096, n // sub),
                                blocks_per_sm=3, **geo) as c:
                t = c.register("mergesort")
                for r0 in range(0, n, sub):
                    o = r0 * 4
                    c.spawn(t, G.gtap_mergesort_args(src.data_ptr() + o, dst.data_ptr() + o, tmp.data_ptr() + o,
                                                     sub, 4096, 65536))
                c.run()
                st = c.stats()
                # block-loop phase cycles per block (acquire, task bodies, post-step, idle), in ms at the max SM clock
                ph = [st[k] / st["n_workers"] / 2.07e6 for k in ("cycles_pop", "cycles_exec", "cycles_push", "cycles_idle")]
                print("mergesort", n, sub, st["kernel_ms"], "phases_ms acquire %.3f body %.3f post %.3f idle %.3f" % tuple(ph))
        out = dst.cpu().numpy().view(np.uint32).reshape(-1, sub)
        assert np.all(out[:, 1:] >= out[:, :-1])
    elif args.case == "kclique":
        n, e = inputs.rmat_graph(args.n or 16, 16, seed=7)
        g = runner.DeviceGraph(n, e)
        for _ in range(args.reps):
            r = runner.kclique(g, args.k, n_queues=args.queues, route=args.route)
            print("kclique", r.values, r.stats["kernel_ms"])
    elif args.case == "fmm":
        n = 1 << (args.n or 18)
        pos, q = inputs.fmm_points(n, args.dist, seed=3)
        with runner.Fmm(order=6, leaf_size=64, theta=0.5, mixed=bool(args.mixed)) as f:
            for _ in range(args.reps):
                f.run(pos, q)
                print("fmm", n, args.dist, f.info())
    elif args.case == "bintree":
        for _ in range(args.reps):
            r = runner.bintree(args.n or 20, args.iters, args.K, route=args.route, block=bool(args.block),
                               n_queues=args.queues, **geo)
            print("bintree", r.values, r.stats["kernel_ms"])
    else:
        print(f"case {args.case} is not available", file=sys.stderr)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main())
