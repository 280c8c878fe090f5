"""The allocation-free sort entry point, through the C ABI.

gsr_sort_pairs_u32_noalloc serves callers that cannot allocate device memory (a step being
recorded into a CUDA graph, a fixed-footprint loop, code inside another allocator's callback);
its scratch is a static device array inside the library. Its output must equal that of
gsr_sort_pairs_u32 (which grows a context workspace) bit for bit, on consecutive calls that
share the static scratch. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2507_23006_gb300 import native

pytestmark = pytest.mark.gpu

MAX_N = 1 << 18


def _noalloc(keys, vals, begin_bit, end_bit, err):
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    st = native.load().gsr_sort_pairs_u32_noalloc(keys.data_ptr(), vals.data_ptr(), ko.data_ptr(), vo.data_ptr(),
                                                  keys.numel(), begin_bit, end_bit, err.data_ptr(),
                                                  torch.cuda.current_stream().cuda_stream)
    return st, ko, vo


@pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")
def test_noalloc_sort_matches_workspace_sort_twice():
    ctx = native.Context(0)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(17)
    for n, bits in ((MAX_N, 32), (100_003, 13)):
        keys = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
        keys[: n // 8] = keys[n // 2]  # repeated keys make the order depend on stability
        kt = torch.from_numpy(keys.view(np.int32)).cuda()
        vt = torch.from_numpy(np.arange(n, dtype=np.int32)).cuda()
        st, ko, vo = _noalloc(kt, vt, 0, bits, err)
        assert st == 0
        kr, vr = native.sort_pairs_u32(ctx, kt, vt, 0, bits)
        torch.cuda.synchronize()
        assert torch.equal(ko, kr) and torch.equal(vo, vr)
    assert int(err.item()) == 0
    # beyond the stated maximum the call refuses without touching the GPU
    big = torch.zeros(MAX_N + 1, dtype=torch.int32, device="cuda")
    st, _, _ = _noalloc(big, big.clone(), 0, 32, err)
    assert st == -5
