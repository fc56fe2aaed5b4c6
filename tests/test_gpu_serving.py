"""Served mode: a resident kernel fed through the inbox; each result equals the result alone (GPU)."""
import time

import numpy as np
import pytest

import oracle
from paper_2604_05982_gb300 import gtap as G
from paper_2604_05982_gb300 import inputs, runner

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _drain(ctx, want, deadline_s=60.0):
    got = {}
    t0 = time.time()
    while len(got) < want:
        for req, r0, r1, st in G.gtap_poll(ctx):
            assert st == 0
            got[req] = r0
        assert time.time() - t0 < deadline_s, f"only {len(got)} of {want} completions"
    return got


def test_served_mix_matches_oracle_and_overlaps():
    graphs = {s: inputs.rmat_graph(s, 16, seed=100 + s) for s in (8, 9, 10)}
    dgs = {s: runner.DeviceGraph(*graphs[s]) for s in graphs}
    with runner.Context(G.GTAP_MODE_THREAD, 4, pool_bytes=1 << 30, scratch_bytes=1 << 28, max_roots=256) as c:
        t_fib, t_nq, t_uts, t_kc = (c.register(p) for p in ("fib", "nqueens", "uts", "kclique"))
        G.gtap_serve_start(c.ctx)
        want = {}
        rng = np.random.default_rng(1)
        for i in range(300):
            kind = i % 4
            if kind == 0:
                n = int(rng.integers(15, 25))
                args, expect = G.gtap_fib_args(n, 1), oracle.fib(n)[0]
                t = t_fib
            elif kind == 1:
                n = int(rng.integers(6, 11))
                args, expect = G.gtap_nqueens_args(n, 1), oracle.nqueens(n)[0]
                t = t_nq
            elif kind == 2:
                rc = int(rng.integers(10, 300))
                args = G.gtap_uts_args(i, runner.UTS_THRESHOLD_Q0199, rc, 5, 1, 0)
                nodes, leaves = oracle.uts(i, rc, 5)
                expect = (nodes << 32) | leaves
                t = t_uts
            else:
                s = (8, 9, 10)[i % 3]
                args, expect = dgs[s].args(4), oracle.kclique(*graphs[s], 4)
                t = t_kc
            req = None
            while req is None:   # the inbox may be momentarily full
                req = G.gtap_submit(c.ctx, t, args, i % 4)
            want[req] = expect
        got = _drain(c.ctx, len(want))
        assert G.gtap_serve_stop(c.ctx, 30000) == 0
        assert got == want


def test_serve_stop_with_nothing_submitted():
    with runner.Context(G.GTAP_MODE_THREAD, 1, max_roots=64) as c:
        c.register("fib")
        G.gtap_serve_start(c.ctx)
        assert G.gtap_serve_stop(c.ctx, 30000) == 0
        # the context runs ordinary batches afterwards
        t = c.register("fib")
        h = c.spawn(t, G.gtap_fib_args(20, 0))
        c.run()
        assert c.result_i64(h) == 6765
