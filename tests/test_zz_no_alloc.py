"""The allocation-free mergesort entry point gives the regular entry point's output.

Callers that cannot allocate device memory (code running during another
framework's CUDA-graph capture, fixed-budget real-time paths, plugins that own
no memory) use gtap_mergesort_noalloc, whose working memory is a fixed device
array inside the library.  This file is collected last so that a run stopping
at the first failure has already run every other test.
"""
import numpy as np
import pytest

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


def test_noalloc_rejects_more_keys_than_its_array_holds():
    src = torch.zeros(16, dtype=torch.int32, device="cuda")
    status = G.gtap_mergesort_noalloc(src.data_ptr(), src.data_ptr(), (1 << 20) + 1, 0, raise_on_error=False)
    assert status == G.GTAP_ERR_INVALID_ARG
