"""Failure detection on its error paths (GPU).

Every failure here is made on the host side or by a bound the kernel checks
itself (a deadline, the host abort word, a capacity): the kernel records an
error status, drains and returns, so the context stays usable.  Nothing traps
or faults the GPU.  Sec. 4: capacity exhaustion and other runtime failures
abort execution with a structured error report.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2604_05982_gb300 import gtap as G
from paper_2604_05982_gb300 import inputs, runner

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _fib10_runs(c, t):
    c.clear()
    h = c.spawn(t, G.gtap_fib_args(10, 0))
    assert c.run() == 0 and c.result_i64(h) == 55


def test_device_deadline_reports_timeout_and_context_recovers():
    # a 2 us device deadline cannot cover fib(30) (2.7 M tasks): the first idle
    # deadline check raises GTAP_ERR_TIMEOUT and every warp drains
    with runner.Context(G.GTAP_MODE_THREAD, 1, timeout_ns=2000) as c:
        t = c.register("fib")
        c.spawn(t, G.gtap_fib_args(30, 0))
        status = c.run(raise_on_error=False)
        assert status == G.GTAP_ERR_TIMEOUT
        err = c.last_error()
        assert err.code == G.GTAP_ERR_TIMEOUT and err.detail == 2000
        G.gtap_set_timeout(c.ctx, 0)   # back to the default deadline
        _fib10_runs(c, t)


def test_host_wait_timeout_raises_abort_word_and_context_recovers():
    # eight chains (m = 1, continuation probability 1 - 2^-20): about 2^20
    # dependent levels each, far more than the 20 ms the host waits
    with runner.Context(G.GTAP_MODE_THREAD, 1) as c:
        t = c.register("uts")
        c.spawn(t, G.gtap_uts_args(5, 2 ** 64 - 2 ** 44, 8, 1, 0, 0))
        G.gtap_run(c.ctx)
        t0 = time.time()
        status = G.gtap_wait(c.ctx, 20, raise_on_error=False)
        assert status == G.GTAP_ERR_TIMEOUT
        assert time.time() - t0 < 10.0          # drained through the mapped abort word
        assert c.last_error().code == G.GTAP_ERR_TIMEOUT
        snap = G.gtap_debug_snapshot(c.ctx)
        assert snap["abort"] == 1 and snap["roots_remaining"] == 1
        t2 = c.register("fib")
        _fib10_runs(c, t2)


def test_served_session_with_exhausted_scratch_reports_error_and_stops():
    # K_1500 oriented by id: first-level candidate sets of up to 1498 vertices need
    # two 4 KiB scratch blocks each; a 64 KiB scratch arena has 15
    n = 1500
    iu, ju = np.triu_indices(n, k=1)
    g = runner.DeviceGraph(n, np.stack([iu, ju], axis=1).astype(np.int32))
    with runner.Context(G.GTAP_MODE_THREAD, 1, scratch_bytes=64 << 10, max_roots=64) as c:
        t = c.register("kclique")
        t_fib = c.register("fib")
        G.gtap_serve_start(c.ctx)
        assert G.gtap_submit(c.ctx, t, g.args(4), 0) is not None
        status, t0 = None, time.time()
        while status is None:
            try:
                assert G.gtap_poll(c.ctx) == []
            except G.GtapError as exc:
                status = exc.status
            assert time.time() - t0 < 30.0, "the session did not report the failure"
        assert status == G.GTAP_ERR_TASK_FAILED
        stop = G.load_library().gtap_serve_stop(c.ctx, 30000)
        assert stop == G.GTAP_ERR_TASK_FAILED
        assert c.last_error().code == G.GTAP_ERR_TASK_FAILED
        # the context runs ordinary batches afterwards
        h = c.spawn(t_fib, G.gtap_fib_args(20, 0))
        assert c.run() == 0 and c.result_i64(h) == oracle.fib(20)[0]


def test_caller_owned_device_arena():
    cfg = runner.make_config()
    need = G.gtap_arena_bytes(G.GTAP_MODE_THREAD, 2, 256 << 20, cfg)
    assert need > 256 << 20
    arena = torch.full((need + 4096,), 0x5A, dtype=torch.uint8, device="cuda")
    base = (arena.data_ptr() + 255) // 256 * 256
    torch.cuda.synchronize()
    with runner.Context(G.GTAP_MODE_THREAD, 2, pool_bytes=256 << 20, device_arena=base, arena_bytes=need) as c:
        t_nq = c.register("nqueens")
        t_fib = c.register("fib")
        h1 = c.spawn(t_nq, G.gtap_nqueens_args(11, 1))
        h2 = c.spawn(t_fib, G.gtap_fib_args(25, 1))
        for _ in range(2):
            c.run()
            assert c.result_u64(h1) == oracle.nqueens(11)[0]
            assert c.result_i64(h2) == oracle.fib(25)[0]
    # the runtime's storage lived in the caller's buffer
    torch.cuda.synchronize()
    assert int((arena != 0x5A).sum()) > 0
    # one byte short is refused
    with pytest.raises(G.GtapError) as exc:
        runner.Context(G.GTAP_MODE_THREAD, 2, pool_bytes=256 << 20, device_arena=base, arena_bytes=need - 1)
    assert exc.value.status == G.GTAP_ERR_NO_MEMORY
