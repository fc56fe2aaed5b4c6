"""Thread-mode parity: every result bit-exact against the oracle (GPU)."""
import struct

import pytest

import oracle
from paper_2604_05982_gb300 import gtap as G
from paper_2604_05982_gb300 import runner

pytestmark = pytest.mark.gpu


def test_fib_small_values():
    ns = list(range(0, 21))
    r = runner.fib(ns)
    assert r.values == [oracle.fib(n)[0] for n in ns]


@pytest.mark.parametrize("grid", [1, 3, 0])
def test_fib30_geometries(grid):
    # one block of 8 warps, three blocks, and the full persistent grid
    r = runner.fib(30, grid_blocks=grid or None)
    v, tasks = oracle.fib(30)
    assert r.values == [v] == [832040]
    # every task runs one step; every non-leaf task runs a second (continuation) step
    leaves = (tasks + 1) // 2
    assert r.stats["tasks_executed"] == tasks + (tasks - leaves)
    assert r.stats["tasks_created"] == tasks


def test_fib_single_warp():
    r = runner.fib(22, grid_blocks=1, threads_per_block=32)
    assert r.values == [oracle.fib(22)[0]]
    assert r.stats["n_workers"] == 1


@pytest.mark.parametrize("q,route", [(1, 0), (3, 1), (8, 1)])
def test_fib_daq(q, route):
    r = runner.fib(27, n_queues=q, route=route)
    assert r.values == [oracle.fib(27)[0]]


@pytest.mark.parametrize("cutoff", [3, 10, 18])
@pytest.mark.parametrize("q,route", [(1, 0), (3, 1)])
def test_fib_sequential_cutoff(cutoff, q, route):
    # calls below the cutoff run the serial recursion in their lane (Sec. 6.3.2);
    # DAQ routes recursive calls, cutoff leaves and continuations to three queues
    for n in (0, 1, 2, cutoff - 1, cutoff, 27):
        want, tasks = oracle.fib_cutoff(n, cutoff)
        r = runner.fib(n, n_queues=q, route=route, cutoff=cutoff)
        assert r.values == [want], n
        assert r.stats["tasks_created"] == tasks


@pytest.mark.parametrize("depth", [1, 4, 7, 13])
@pytest.mark.parametrize("q,route", [(1, 0), (2, 2), (4, 1)])
def test_nqueens_cutoff_depth(depth, q, route):
    # boards with `depth` rows placed finish their search serially (Sec. 6.3.1 uses 7)
    sols, tasks = oracle.nqueens_cutoff(13, depth)
    r = runner.nqueens(13, n_queues=q, route=route, cutoff=depth)
    assert r.values == [sols] == [73712]
    assert r.stats["tasks_created"] == tasks


@pytest.mark.parametrize("n", list(range(1, 12)))
def test_nqueens_small(n):
    r = runner.nqueens(n)
    sols, tasks = oracle.nqueens(n)
    assert r.values == [sols]
    assert r.stats["tasks_created"] == tasks


@pytest.mark.parametrize("q", [1, 2, 4, 8])
def test_nqueens13_daq(q):
    r = runner.nqueens(13, n_queues=q, route=1 if q > 1 else 0)
    sols, tasks = oracle.nqueens(13)
    assert r.values == [sols] == [73712]
    assert r.stats["tasks_created"] == tasks


def test_uts_seed42():
    r = runner.uts(42)
    assert r.values == [oracle.uts(42)]


@pytest.mark.parametrize("seed,rc,m,thr", [(1, 50, 3, 2 ** 62), (7, 10, 2, 2 ** 63 - 2 ** 60), (5, 1, 1, 0),
                                          (42, 0, 5, 2 ** 63), (3, 100, 1, 2 ** 64 - 2 ** 58)])
def test_uts_variants(seed, rc, m, thr):
    r = runner.uts(seed, rc, m, thr)
    assert r.values == [oracle.uts(seed, rc, m, thr)]


def test_uts_daq_three_queues():
    r = runner.uts(42, n_queues=3, route=1)
    assert r.values == [oracle.uts(42)]


def test_integrate_thread_bit_exact():
    for a, b, eps in [(-1.0, 1.0, 1e-10), (0.0, 1.0, 1e-8), (0.25, 0.5, 1e-12)]:
        r = runner.integrate(a, b, eps)
        want, _ = oracle.integrate_thread(a, b, eps)
        assert struct.pack("<d", r.values[0]) == struct.pack("<d", want)


def test_batched_roots_mixed_sizes():
    ns = [30, 5, 25, 1, 0, 28, 17] * 9
    r = runner.fib(ns)
    assert r.values == [oracle.fib(n)[0] for n in ns]


def test_repeated_runs_reuse_context():
    with runner.Context(G.GTAP_MODE_THREAD, 4) as c:
        t = c.register("nqueens")
        h = c.spawn(t, G.gtap_nqueens_args(10, 1))
        for _ in range(3):
            c.run()
            assert c.result_u64(h) == 724


def test_pool_exhaustion_reports_error():
    with runner.Context(G.GTAP_MODE_THREAD, 1, pool_bytes=64 * 1024, grid_blocks=1) as c:
        t = c.register("fib")
        c.spawn(t, G.gtap_fib_args(25, 0))
        status = c.run(raise_on_error=False)
        assert status == G.GTAP_ERR_POOL_EXHAUSTED
        assert c.last_error().code == G.GTAP_ERR_POOL_EXHAUSTED
        # the context stays usable after the error
        c.clear()
        h = c.spawn(t, G.gtap_fib_args(10, 0))
        assert c.run() == 0 and c.result_i64(h) == 55


def test_deque_overflow_reports_error():
    with runner.Context(G.GTAP_MODE_THREAD, 1, deque_capacity=32, grid_blocks=1, threads_per_block=32) as c:
        t = c.register("nqueens")
        c.spawn(t, G.gtap_nqueens_args(12, 0))
        status = c.run(raise_on_error=False)
        assert status == G.GTAP_ERR_DEQUE_OVERFLOW


def test_graph_replay_same_results_and_reset():
    with runner.Context(G.GTAP_MODE_THREAD, 4) as c:
        t = c.register("nqueens")
        hs = [c.spawn(t, G.gtap_nqueens_args(n, 1)) for n in (6, 9, 11, 12)]
        c.capture()
        for _ in range(4):
            c.run()
            assert [c.result_u64(h) for h in hs] == [oracle.nqueens(n)[0] for n in (6, 9, 11, 12)]
            assert c.stats()["kernel_ms"] > 0 and c.stats()["run_ms"] >= c.stats()["kernel_ms"]
        # a new root drops the graph; the next run is a plain launch with the new batch
        h2 = c.spawn(t, G.gtap_nqueens_args(8, 1))
        c.run()
        assert c.result_u64(h2) == 92 and c.result_u64(hs[1]) == 352


@pytest.mark.parametrize("n,sc,mc", [(1, 64, 256), (64, 64, 256), (1000, 64, 256), (100_003, 64, 256),
                                     (1 << 20, 64, 256), (50_000, 16, 1), (77_777, 256, 4096)])
@pytest.mark.parametrize("q,route", [(1, 0), (3, 1)])
def test_cilksort_thread_mode(n, sc, mc, q, route):
    # thread-mode Cilksort (Sec. 6.3), DAQ with recursive / serial-sort / serial-merge queues
    import numpy as np
    import torch
    from paper_2604_05982_gb300 import inputs
    keys = inputs.keys_u32(n, seed=7)
    keys[: n // 7] = keys[0]        # runs of equal keys
    src = torch.from_numpy(keys.view(np.int32)).cuda()
    dst = torch.full_like(src, -1)
    tmp = torch.empty_like(src)
    torch.cuda.synchronize()
    r = runner.cilksort_ptrs(src.data_ptr(), dst.data_ptr(), tmp.data_ptr(), n, sc, mc, n_queues=q, route=route,
                             pool_bytes=1 << 30)
    want, tasks = oracle.cilksort(keys, sc, mc)
    assert np.array_equal(dst.cpu().numpy().view(np.uint32), want)
    assert r.stats["tasks_created"] == tasks
    # in place (src == dst)
    runner.cilksort_ptrs(src.data_ptr(), src.data_ptr(), tmp.data_ptr(), n, sc, mc, pool_bytes=1 << 30)
    assert np.array_equal(src.cpu().numpy().view(np.uint32), want)
