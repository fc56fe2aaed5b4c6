"""Autotuner (gtap_autotune): every trial reproduces the oracle's answer and the
chosen configuration is the fastest trial seen along the descent (GPU)."""
import numpy as np
import pytest

import oracle
from paper_2604_05982_gb300 import gtap as G
from paper_2604_05982_gb300 import inputs, runner

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _check(best, trials):
    assert trials and all(t["status"] == 0 for t in trials), trials
    ok = [t["kernel_ms"] for t in trials]
    assert best["kernel_ms"] == min(ok) or best["kernel_ms"] <= ok[0]
    assert best["blocks_per_sm"] >= 1 and best["deque_capacity"] in (1024, 4096, 16384)


def test_autotune_thread_mode_nqueens_batch():
    args = [G.gtap_nqueens_args(n, 1) for n in (9, 10, 11)]
    best, trials = G.gtap_autotune(G.GTAP_MODE_THREAD, "nqueens", args, 256 << 20, runner.make_config(), reps=2)
    _check(best, trials)
    # start + blocks/SM 4 + steal 3 + queues 3 + capacity 2 + idle back-off 2
    assert len(trials) == 1 + 4 + 3 + 3 + 2 + 2
    assert best["idle_backoff_ns"] in (512, 2048, 8192)
    # the tuned configuration still gives the oracle's counts
    with runner.Context(G.GTAP_MODE_THREAD, best["n_queues"], pool_bytes=256 << 20,
                        blocks_per_sm=best["blocks_per_sm"], deque_capacity=best["deque_capacity"],
                        steal_policy=best["steal_policy"], idle_backoff_ns=best["idle_backoff_ns"]) as c:
        t = c.register("nqueens")
        hs = [c.spawn(t, a) for a in args]
        c.run()
        assert [c.result_u64(h) for h in hs] == [oracle.nqueens(n)[0] for n in (9, 10, 11)]


def test_autotune_block_mode_mergesort():
    n = 1 << 20
    keys = inputs.keys_u32(n, seed=2)
    src = torch.from_numpy(keys.view(np.int32)).cuda()
    dst = torch.empty_like(src)
    tmp = torch.empty_like(src)
    torch.cuda.synchronize()
    a = G.gtap_mergesort_args(src.data_ptr(), dst.data_ptr(), tmp.data_ptr(), n, 4096, 16384)
    best, trials = G.gtap_autotune(G.GTAP_MODE_BLOCK, "mergesort", [a], 256 << 20, runner.make_config(), reps=2)
    _check(best, trials)
    assert np.array_equal(dst.cpu().numpy().view(np.uint32), oracle.sort_u32(keys))


def test_autotune_with_fixed_queues_keeps_them():
    args = [G.gtap_nqueens_args(10, 1)]
    best, trials = G.gtap_autotune(G.GTAP_MODE_THREAD, "nqueens", args, 256 << 20, runner.make_config(), reps=1,
                                   n_queues=4, tune_mask=G.GTAP_TUNE_BLOCKS | G.GTAP_TUNE_STEAL)
    _check(best, trials)
    assert len(trials) == 1 + 4 + 3
    assert all(t["n_queues"] == 4 and t["deque_capacity"] == 4096 for t in trials)


def test_autotune_rejects_bad_arguments():
    with pytest.raises(G.GtapError):
        G.gtap_autotune(G.GTAP_MODE_THREAD, "no_such_program", [G.gtap_fib_args(10, 0)], 1 << 24)
    with pytest.raises(G.GtapError):
        G.gtap_autotune(G.GTAP_MODE_BLOCK, "mergesort", [G.gtap_fib_args(10, 0)], 1 << 24, n_queues=2)
