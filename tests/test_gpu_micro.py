"""Mode/DAQ microbenchmark programs and the scheduler comparison variants, bit-exact against the oracle (GPU).

Sec. 6.1 (full binary task tree in thread and block mode, block mode with a
cutoff), Sec. 6.2 (heterogeneous leaves with and without DAQ) and Sec. 6.5
(centralised queue and non-batched stealing against batched stealing).
"""
import pytest

import oracle
from paper_2604_05982_gb300 import gtap as G
from paper_2604_05982_gb300 import runner

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("depth,iters,K", [(0, 3, 1), (1, 0, 1), (5, 1, 2), (12, 37, 1), (12, 16, 4), (16, 2, 3)])
def test_bintree_thread_mode(depth, iters, K):
    want, tasks = oracle.bintree(depth, iters, K)
    r = runner.bintree(depth, iters, K)
    assert r.values == [want]
    assert r.stats["tasks_created"] == tasks


@pytest.mark.parametrize("K", [2, 4])
def test_bintree_daq_routes_leaves_by_function(K):
    want, tasks = oracle.bintree(14, 24, K)
    r = runner.bintree(14, 24, K, route=1, n_queues=K + 1)
    assert r.values == [want]
    assert r.stats["tasks_created"] == tasks


@pytest.mark.parametrize("bs", [32, 128, 256])
@pytest.mark.parametrize("cutoff", [0, 5])
def test_bintree_block_mode(bs, cutoff):
    for depth, iters, K in [(0, 100, 1), (6, 1, 1), (11, 300, 4), (13, 7, 2)]:
        want, tasks = oracle.bintree(depth, iters, K, cutoff=cutoff)
        r = runner.bintree(depth, iters, K, block=True, cutoff=cutoff, threads_per_block=bs)
        assert r.values == [want], (depth, iters, K)
        assert r.stats["tasks_created"] == tasks


def test_bintree_rejects_thread_mode_cutoff():
    with runner.Context(G.GTAP_MODE_THREAD, 1) as c:
        t = c.register("bintree")
        with pytest.raises(G.GtapError):
            c.spawn(t, G.gtap_bintree_args(5, 1, 1, 0, 3, 0))


@pytest.mark.parametrize("sched", [G.GTAP_SCHED_GLOBAL, G.GTAP_SCHED_SINGLE, G.GTAP_SCHED_BATCHED])
@pytest.mark.parametrize("grid", [1, 5, 0])
def test_scheduler_variants_fib(sched, grid):
    v, tasks = oracle.fib(25)
    r = runner.fib(25, scheduler=sched, grid_blocks=grid or None)
    assert r.values == [v]
    assert r.stats["tasks_created"] == tasks


@pytest.mark.parametrize("sched", [G.GTAP_SCHED_GLOBAL, G.GTAP_SCHED_SINGLE])
def test_scheduler_variants_tree_and_batch(sched):
    assert runner.uts(42, scheduler=sched).values == [oracle.uts(42)]
    ns = [22, 3, 0, 18, 25, 1] * 5
    assert runner.fib(ns, scheduler=sched).values == [oracle.fib(n)[0] for n in ns]
    want, _ = oracle.bintree(12, 5, 4)
    assert runner.bintree(12, 5, 4, scheduler=sched).values == [want]


def test_scheduler_variant_needs_a_compiled_program_set():
    # the comparison variants are compiled for fib, the hashed tree and the binary tree
    with runner.Context(G.GTAP_MODE_THREAD, 1, scheduler=G.GTAP_SCHED_GLOBAL) as c:
        t = c.register("nqueens")
        c.spawn(t, G.gtap_nqueens_args(8, 0))
        with pytest.raises(G.GtapError) as exc:
            c.run()
        assert exc.value.status == G.GTAP_ERR_INVALID_ARG
    # and need one queue per warp
    with pytest.raises(G.GtapError):
        runner.Context(G.GTAP_MODE_THREAD, 2, scheduler=G.GTAP_SCHED_SINGLE)
