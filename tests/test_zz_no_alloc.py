"""The allocation-free sort entry point, through the C ABI.

gsr_sort_pairs_u32_noalloc serves callers that cannot allocate device memory: a step being
recorded into a CUDA graph (an allocation cannot be recorded, and cudaMalloc may synchronise the
device), a loop that must keep a fixed memory footprint, or code running inside another
allocator's callback. Its scratch is a static device array inside the library. Its output must
equal that of gsr_sort_pairs_u32 (which grows a context workspace) and numpy's stable argsort, bit
for bit, on consecutive calls that share the static scratch. This file is collected last on
purpose: if it fails, a run that stops at the first failure has already run everything else.
"""
import numpy as np
import pytest
import torch

from paper_2507_23006_gb300 import native

pytestmark = pytest.mark.gpu

MAX_N = 1 << 18


def _noalloc(keys, vals, begin_bit, end_bit, err, ko=None, vo=None):
    ko = torch.empty_like(keys) if ko is None else ko
    vo = torch.empty_like(vals) if vo is None else vo
    st = native.load().gsr_sort_pairs_u32_noalloc(keys.data_ptr(), vals.data_ptr(), ko.data_ptr(), vo.data_ptr(),
                                                  keys.numel(), begin_bit, end_bit,
                                                  None if err is None else err.data_ptr(),
                                                  torch.cuda.current_stream().cuda_stream)
    return st, ko, vo


def _keys(rng, n):
    keys = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    keys[: n // 8] = keys[n // 2]  # repeated keys make the order depend on stability
    return keys


@pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")
def test_noalloc_sort_matches_workspace_sort_and_numpy_twice():
    ctx = native.Context(0)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(17)
    for n, bits in ((MAX_N, 32), (100_003, 13)):
        keys = _keys(rng, n)
        kt = torch.from_numpy(keys.view(np.int32)).cuda()
        vt = torch.from_numpy(np.arange(n, dtype=np.int32)).cuda()
        ko = torch.empty_like(kt)
        vo = torch.empty_like(vt)
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        st, ko, vo = _noalloc(kt, vt, 0, bits, err, ko, vo)
        torch.cuda.synchronize()
        assert st == 0
        assert torch.cuda.memory_allocated() == before  # nothing taken from torch's allocator either
        kr, vr = native.sort_pairs_u32(ctx, kt, vt, 0, bits)
        torch.cuda.synchronize()
        assert torch.equal(ko, kr) and torch.equal(vo, vr)
        order = np.argsort(keys & np.uint32((1 << bits) - 1) if bits < 32 else keys, kind="stable")
        np.testing.assert_array_equal(vo.cpu().numpy(), order.astype(np.int32))
        np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    assert int(err.item()) == 0
    ctx.close()


@pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")
def test_noalloc_sort_arguments():
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    keys = torch.from_numpy(_keys(np.random.default_rng(3), 5000).view(np.int32)).cuda()
    vals = torch.arange(5000, dtype=torch.int32, device="cuda")
    # an empty bit range copies the inputs
    st, ko, vo = _noalloc(keys, vals, 7, 7, err)
    torch.cuda.synchronize()
    assert st == 0 and torch.equal(ko, keys) and torch.equal(vo, vals)
    # without an error word a timeout could not be reported: refused
    st, _, _ = _noalloc(keys, vals, 0, 32, None)
    assert st == -1
    # beyond the stated maximum the call refuses without touching the GPU
    big = torch.zeros(MAX_N + 1, dtype=torch.int32, device="cuda")
    st, _, _ = _noalloc(big, big.clone(), 0, 32, err)
    assert st == -5
    assert int(err.item()) == 0
