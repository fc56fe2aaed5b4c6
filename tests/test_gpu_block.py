"""Block-mode parity: mergesort bit-exact vs the oracle sort; Program 1 block mode bit-exact (GPU)."""
import struct

import numpy as np
import pytest

import oracle
from paper_2604_05982_gb300 import inputs, runner

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sort_on_gpu(keys: np.ndarray, in_place=False, **kw):
    n = keys.size
    src = torch.from_numpy(keys.view(np.int32)).cuda()
    dst = src if in_place else torch.empty_like(src)
    tmp = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    r = runner.mergesort_ptrs(src.data_ptr(), dst.data_ptr(), tmp.data_ptr(), n, **kw)
    out = dst.cpu().numpy().view(np.uint32)
    return out, r


@pytest.mark.parametrize("n", [0, 1, 2, 4095, 4096, 4097, 8192 + 17, 100003, (1 << 20) + 3])
def test_mergesort_sizes(n):
    keys = inputs.keys_u32(n, seed=1)
    out, _ = _sort_on_gpu(keys)
    assert np.array_equal(out, oracle.sort_u32(keys))


def test_mergesort_in_place_and_small_leaf():
    keys = inputs.keys_u32(300001, seed=5)
    out, _ = _sort_on_gpu(keys, in_place=True, leaf=1000, merge_cutoff=2048)
    assert np.array_equal(out, oracle.sort_u32(keys))


def test_mergesort_duplicates_and_extremes():
    keys = (inputs.keys_u32(200000, seed=9) % 7).astype(np.uint32)
    keys[::1000] = 0xFFFFFFFF
    keys[1::1000] = 0
    out, _ = _sort_on_gpu(keys, merge_cutoff=8192)
    assert np.array_equal(out, oracle.sort_u32(keys))


def test_mergesort_2pow26_full_size():
    keys = inputs.keys_u32(1 << 26, seed=1)
    out, r = _sort_on_gpu(keys)
    assert np.all(out[1:] >= out[:-1])
    assert np.array_equal(out, oracle.sort_u32(keys))


@pytest.mark.parametrize("bps", [3, 6])
def test_mergesort_2pow26_bench_launch_configuration(bps):
    # the configuration the bench times: 4096-key leaves, 65536-key merge pieces,
    # the block counts per SM the autotuner picks, rings of 16384
    keys = inputs.keys_u32(1 << 26, seed=1)
    out, _ = _sort_on_gpu(keys, leaf=4096, merge_cutoff=65536, blocks_per_sm=bps, deque_capacity=16384)
    assert np.array_equal(out, oracle.sort_u32(keys))


@pytest.mark.parametrize("grid", [1, 2])
def test_mergesort_small_grid(grid):
    keys = inputs.keys_u32(50000, seed=2)
    out, r = _sort_on_gpu(keys, grid_blocks=grid)
    assert np.array_equal(out, oracle.sort_u32(keys))


@pytest.mark.parametrize("bs", [128, 256])
def test_integrate_block_bit_exact(bs):
    for a, b, eps in [(-1.0, 1.0, 1e-10), (0.0, 1.0, 1e-12)]:
        r = runner.integrate(a, b, eps, block=True, threads_per_block=bs)
        want, _ = oracle.integrate_block(a, b, eps, bs)
        assert struct.pack("<d", r.values[0]) == struct.pack("<d", want)
