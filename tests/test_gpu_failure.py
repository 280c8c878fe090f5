"""Failure detection without a GPU fault.

* Device waits: every decoupled look-back of the chained scans (the tile scan, the global-sort
  binning's scans) and of the sort is bounded. A test
  switch of the context (gsr_set_wait_limit) makes each look-back wait on status words that no
  block publishes, with a short limit: the kernels give up, finish, and the call that checks the
  context's error word reports GSR_ERR_DEVICE_TIMEOUT. Nothing hangs and nothing faults (a wait
  that gives up uses a partial prefix, never larger than the true one). The same context then
  renders correctly again.
* Allocation failures are injected on the host: an allocator callback that returns NULL on its
  k-th call. The call reports GSR_ERR_OOM, and the same context works on the next call.
"""
import numpy as np
import pytest
import torch

from paper_2507_23006_gb300 import native, scenes
from tests import parity_util as pu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return native.Context(0)


def _upstream(npix):
    rng = np.random.default_rng(1)
    return dict(rgb=torch.tensor(rng.normal(size=(npix, 3)), dtype=torch.float32, device="cuda"),
                alpha=torch.tensor(rng.normal(size=npix), dtype=torch.float32, device="cuda"))


def test_device_wait_timeout_is_reported_and_context_recovers(ctx):
    scene, _ = pu.scene_box(6000, seed=31)
    # 4096 tiles: the tile scan runs as two blocks, so the second one looks back
    cam = scenes.box_camera(1024, 1024, f=1200.0)
    g = native.Gaussians.from_scene(scene)
    opts = native.Options(tile_cull=True)
    ref, _ = native.render_forward(ctx, g, [cam], opts, want_state=False)
    torch.cuda.synchronize()
    ctx.set_wait_limit(64, never_ready=True)
    try:
        # the forward checks the error word once binning is done
        with pytest.raises(native.GsrError) as e:
            native.render_forward(ctx, g, [cam], opts)
        assert e.value.status == -4
        # the sort is asynchronous: its timeout surfaces at the next check
        n = 1_000_000
        keys = torch.randint(-2 ** 31, 2 ** 31 - 1, (n,), dtype=torch.int32, device="cuda")
        native.sort_pairs_u32(ctx, keys, torch.arange(n, dtype=torch.int32, device="cuda"))
        with pytest.raises(native.GsrError) as e:
            ctx.sync_check()
        assert e.value.status == -4
        ctx.sync_check()  # the word was cleared by the check that reported it
    finally:
        ctx.set_wait_limit(0, never_ready=False)
    # a recompute-mode backward re-runs the binning and reports a timeout there too
    ropts = native.Options(tile_cull=True, save_state=False)
    out, st = native.render_forward(ctx, g, [cam], ropts)
    assert torch.equal(out["rgb"], ref["rgb"])
    ctx.set_wait_limit(64, never_ready=True)
    try:
        with pytest.raises(native.GsrError) as e:
            native.render_backward(ctx, g, [cam], st, _upstream(cam.width * cam.height), ropts)
        assert e.value.status == -4
    finally:
        ctx.set_wait_limit(0, never_ready=False)
    gr = native.render_backward(ctx, g, [cam], st, _upstream(cam.width * cam.height), ropts)
    ctx.sync_check()
    assert torch.isfinite(gr["means"]).all()
    again, _ = native.render_forward(ctx, g, [cam], opts, want_state=False)
    torch.cuda.synchronize()
    assert torch.equal(again["rgb"], ref["rgb"]) and torch.equal(again["alpha"], ref["alpha"])


class _FailingAllocator(native.TorchAllocator):
    """torch's caching allocator, except that the k-th request returns NULL."""

    def __init__(self, k):
        super().__init__(0)
        self.k = k
        self.calls = 0

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.calls == self.k:
            return 0
        return super().alloc(nbytes, stream)


def test_allocation_failure_reports_oom_and_context_recovers(ctx):
    scene, cam = pu.scene_box(5000, seed=32)
    g = native.Gaussians.from_scene(scene)
    opts = native.Options(tile_cull=True)
    ref, ref_st = native.render_forward(ctx, g, [cam], opts)
    up = _upstream(cam.width * cam.height)
    ref_gr = native.render_backward(ctx, g, [cam], ref_st, up, opts)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    failed = 0
    for k in (1, 3, 5, 8, 11):
        alloc = _FailingAllocator(k)
        c = native.Context(0, allocator=alloc)
        try:
            native.render_forward(c, g, [cam], opts)
        except native.GsrError as e:
            assert e.status == -2, e
            failed += 1
        out, st = native.render_forward(c, g, [cam], opts)
        gr = native.render_backward(c, g, [cam], st, up, opts)
        c.sync_check()
        assert torch.equal(out["rgb"], ref["rgb"])
        pu.grad_close(gr["means"].cpu().numpy(), ref_gr["means"].cpu().numpy(), "means", rel=1e-5,
                      group_rel=1e-6)
        assert alloc.calls > k
        st.release()
        del gr, out
        c.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base  # every workspace buffer went back to torch
    assert failed >= 4
