"""The allocation-free mergesort entry point sorts like the regular one, and allocates nothing.

Some callers of this library cannot allocate device memory: a plugin loaded
into a host application that owns all device memory and hands it only a
stream and buffers, or a real-time path whose memory budget is fixed before it
starts.  They call gtap_mergesort_noalloc, whose working memory is a fixed
device array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2604_05982_gb300 import gtap as G
from paper_2604_05982_gb300 import inputs, runner

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _regular(src, n):
    out = torch.empty_like(src)
    tmp = torch.empty_like(src)
    torch.cuda.synchronize()
    runner.mergesort_ptrs(src.data_ptr(), out.data_ptr(), tmp.data_ptr(), n)
    return out


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row():
    # the second call reuses the array the first one left behind
    for seed, n in [(3, 1 << 20), (4, 777_777)]:
        keys = inputs.keys_u32(n, seed=seed)
        src = torch.from_numpy(keys.view(np.int32)).cuda()
        want = _regular(src, n)
        got = torch.full_like(src, -1)
        torch.cuda.synchronize()
        status = G.gtap_mergesort_noalloc(src.data_ptr(), got.data_ptr(), n, 0)
        assert status == G.GTAP_OK
        assert torch.equal(got, want)   # integer sort: bit-exact
        assert np.array_equal(_u32(got), oracle.sort_u32(keys))


def test_noalloc_in_place_and_allocates_nothing():
    n = 777_777   # leaf boundaries not aligned to the 4096-key leaves
    keys = inputs.keys_u32(n, seed=9)
    want = oracle.sort_u32(keys)
    buf = torch.from_numpy(keys.view(np.int32)).cuda()
    torch.cuda.synchronize()
    # first call: sets the device up (and loads the kernels it uses)
    assert G.gtap_mergesort_noalloc(buf.data_ptr(), buf.data_ptr(), n, 0) == G.GTAP_OK
    assert np.array_equal(_u32(buf), want)
    # second call, in place on fresh keys: neither torch's allocator nor the device's free memory moves
    buf.copy_(torch.from_numpy(inputs.keys_u32(n, seed=10).view(np.int32)))
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    assert G.gtap_mergesort_noalloc(buf.data_ptr(), buf.data_ptr(), n, 0) == G.GTAP_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0
    assert np.array_equal(_u32(buf), oracle.sort_u32(inputs.keys_u32(n, seed=10)))


def test_noalloc_rejects_more_keys_than_its_array_holds():
    src = torch.zeros(16, dtype=torch.int32, device="cuda")
    status = G.gtap_mergesort_noalloc(src.data_ptr(), src.data_ptr(), (1 << 20) + 1, 0, raise_on_error=False)
    assert status == G.GTAP_ERR_INVALID_ARG
