"""Continuous-batching render server: resident scenes with detail levels, per-view level
selection under a Gaussian budget (Sec. 3.4.2), memory-admitted slots whose work overlaps on
the GPU.

A request is (scene, camera). On submission the host picks a level per partition for that
view (gsr_select_lod: invisible partitions culled, nearer partitions finer, farthest demoted
first while over the budget) and estimates the device memory the render needs
(gsr_workspace_query plus the output images). Each slot owns a library context and a CUDA
stream and is driven by its own host thread; a free slot takes the oldest waiting request as
soon as the memory it needs is free, together with later waiting requests of the same scene, up
to `max_batch` views of any resolutions and detail selections in one launch: the launch renders
the union of their selected segments, each segment marked with the views that selected it
(gsr_gaussians.seg_cams), and each view's image is the one it gets alone. The batch's memory is
that of the union. Slots run concurrently, so requests that arrive while others render are
admitted as slots and memory free up. Latency is arrival to image ready.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Optional

import numpy as np
import torch

from . import native
from .lod import LodScene


@dataclasses.dataclass
class Request:
    rid: int
    scene: str
    camera: object
    t_arrival: float
    segments: list = None
    selection: list = None  # (partition, level, begin, count) of each selected partition
    n_selected: int = 0
    over_budget: bool = False
    mem_bytes: int = 0
    t_start: Optional[float] = None
    t_done: Optional[float] = None
    rgb: Optional[torch.Tensor] = None
    error: Optional[str] = None
    batch_size: int = 0
    done: threading.Event = dataclasses.field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class _Resident:
    def __init__(self, lod: LodScene, device: str, attr_dtype, sh_dtype):
        self.lod = lod
        self.g = native.Gaussians.from_scene(lod.gaussians, device=device, attr_dtype=attr_dtype, sh_dtype=sh_dtype)


class RenderServer:
    def __init__(self, device: int = 0, slots: int = 4, memory_budget: Optional[int] = None,
                 gaussian_budget: int = 4_000_000, thresholds=(100.0, 200.0), max_batch: int = 8,
                 opts: Optional[native.Options] = None, keep_results: bool = True):
        self.device = int(device)
        self.dev = f"cuda:{self.device}"
        torch.cuda.set_device(self.device)
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            memory_budget = int(0.5 * free)
        self.memory_budget = int(memory_budget)
        self.gaussian_budget = int(gaussian_budget)
        self.thresholds = tuple(float(t) for t in thresholds)
        self.max_batch = int(max_batch)
        # keep_results=False drops each image once it is ready (a server hands it to its
        # client); kept, every image of a long trace stays in device memory
        self.keep_results = bool(keep_results)
        self.opts = opts or native.Options(tile_cull=True, save_state=False)
        self.scenes: dict[str, _Resident] = {}
        self.queue: collections.deque = collections.deque()
        self.cv = threading.Condition()
        self.mem_in_use = 0
        self.in_flight = 0
        self.max_in_flight = 0
        self.running = True
        self._next_id = 0
        self._slots = [(native.Context(self.device), torch.cuda.Stream(self.device)) for _ in range(slots)]
        self._threads = [threading.Thread(target=self._worker, args=(k,), daemon=True) for k in range(slots)]
        for t in self._threads:
            t.start()

    # ---- scenes and requests ---------------------------------------------------------------

    def add_scene(self, name: str, lod: LodScene, attr_dtype=torch.float16, sh_dtype=torch.float16):
        self.scenes[name] = _Resident(lod, self.dev, attr_dtype, sh_dtype)

    def select(self, scene: str, cam):
        segs, nsel, over, _ = self.select_levels(scene, cam)
        return segs, nsel, over

    def select_levels(self, scene: str, cam):
        """Level selection of one view -> (segments, n_selected, over budget, selection), the
        selection listing (partition, level, begin, count) in partition order."""
        r = self.scenes[scene]
        st, levels, segs, nsel = native.select_lod(r.lod.aabb, r.lod.level_offsets, cam, self.thresholds,
                                                   self.gaussian_budget)
        lo = r.lod.level_offsets
        sel = []
        for p, lev in enumerate(levels):
            if lev >= 0 and lo[lev, p + 1] > lo[lev, p]:
                sel.append((p, int(lev), int(lo[lev, p]), int(lo[lev, p + 1] - lo[lev, p])))
        assert [(b, c) for _, _, b, c in sel] == [tuple(x) for x in segs]
        return segs, nsel, st == native.GSR_WARN_OVER_BUDGET, sel

    def _memory(self, n_render: int, cams) -> int:
        """Device memory of one launch: the library's workspace and the output images."""
        ctx0 = self._slots[0][0]
        n = max(int(n_render), 1)
        return ctx0.workspace_query(n, list(cams), 3 * n) + sum(c.width * c.height for c in cams) * 6 * 4

    def submit(self, scene: str, cam, t_arrival: Optional[float] = None) -> Request:
        segs, nsel, over, sel = self.select_levels(scene, cam)
        mem = self._memory(nsel, [cam])
        with self.cv:
            req = Request(self._next_id, scene, cam, time.perf_counter() if t_arrival is None else t_arrival,
                          segs, sel, nsel, over, mem)
            self._next_id += 1
            if mem > self.memory_budget:
                req.error = "request needs more memory than the server's budget"
                req.t_done = time.perf_counter()
                req.done.set()
                return req
            self.queue.append(req)
            self.cv.notify_all()
        return req

    def close(self):
        with self.cv:
            self.running = False
            self.cv.notify_all()
        for t in self._threads:
            t.join(timeout=10)
        for ctx, _ in self._slots:
            ctx.close()

    # ---- slots ------------------------------------------------------------------------------

    def _take(self):
        """Under the lock: the oldest waiting request if its memory fits, plus later waiting
        requests of the same scene (any resolution, any level selection) while the memory of
        the batch (the union of their selections, all their cameras) fits: one launch."""
        if not self.queue:
            return None
        head = self.queue[0]
        if self.mem_in_use + head.mem_bytes > self.memory_budget:
            return None
        batch = [self.queue.popleft()]
        mem = head.mem_bytes
        union = {(p, lev): cnt for p, lev, _, cnt in head.selection}
        keep = collections.deque()
        while self.queue and len(batch) < self.max_batch:
            r = self.queue.popleft()
            if r.scene != head.scene:
                keep.append(r)
                continue
            grown = dict(union)
            grown.update({(p, lev): cnt for p, lev, _, cnt in r.selection})
            need = self._memory(sum(grown.values()), [q.camera for q in batch] + [r.camera])
            if self.mem_in_use + need <= self.memory_budget:
                batch.append(r)
                union, mem = grown, need
            else:
                keep.append(r)
        self.queue.extendleft(reversed(keep))
        self.mem_in_use += mem
        self.in_flight += len(batch)
        self.max_in_flight = max(self.max_in_flight, self.in_flight)
        return batch, mem

    def _worker(self, k: int):
        ctx, stream = self._slots[k]
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                taken = None
                while self.running and (taken := self._take()) is None:
                    self.cv.wait(timeout=0.05)
                if not self.running and taken is None:
                    return
            batch, mem = taken
            t0 = time.perf_counter()
            try:
                res = self.scenes[batch[0].scene]
                if len(batch) == 1:
                    g = dataclasses.replace(res.g, segments=batch[0].segments)
                else:
                    segs, masks = native.union_segments([r.selection for r in batch])
                    g = dataclasses.replace(res.g, segments=segs, segment_cams=masks)
                cams = [r.camera for r in batch]
                with torch.cuda.stream(stream):
                    out, _ = native.render_forward(ctx, g, cams, self.opts, want_state=False, stream=stream)
                stream.synchronize()
                t1 = time.perf_counter()
                off = 0
                for r in batch:
                    hw = r.camera.width * r.camera.height
                    if self.keep_results:
                        r.rgb = out["rgb"][off:off + hw].view(r.camera.height, r.camera.width, 3)
                    off += hw
                    r.t_start, r.t_done, r.batch_size = t0, t1, len(batch)
                del out
            except Exception as e:  # reported on the request, the slot keeps serving
                for r in batch:
                    r.error = str(e)
                    r.t_done = time.perf_counter()
            with self.cv:
                self.mem_in_use -= mem
                self.in_flight -= len(batch)
                self.cv.notify_all()
            for r in batch:
                r.done.set()

    # ---- traces -----------------------------------------------------------------------------

    def run_trace(self, trace, timeout: float = 600.0) -> dict:
        """trace: list of (seconds after start, scene, camera), sorted by time. Submits each at its
        time and waits for all. Returns the requests and latency / throughput statistics."""
        t0 = time.perf_counter()
        reqs = []
        for t_rel, scene, cam in trace:
            now = time.perf_counter() - t0
            if t_rel > now:
                time.sleep(t_rel - now)
            reqs.append(self.submit(scene, cam, t_arrival=t0 + t_rel))
        for r in reqs:
            r.done.wait(timeout)
        t_end = max((r.t_done for r in reqs if r.t_done is not None), default=t0)
        ok = [r for r in reqs if r.error is None and r.t_done is not None]
        lat = np.array([r.latency for r in ok]) * 1e3
        return dict(requests=reqs, served=len(ok), failed=len(reqs) - len(ok),
                    p50_ms=float(np.percentile(lat, 50)) if lat.size else None,
                    p99_ms=float(np.percentile(lat, 99)) if lat.size else None,
                    mean_ms=float(lat.mean()) if lat.size else None,
                    fps=len(ok) / max(t_end - t0, 1e-9),
                    max_in_flight=self.max_in_flight,
                    mean_batch=float(np.mean([r.batch_size for r in ok])) if ok else 0.0,
                    mean_selected=float(np.mean([r.n_selected for r in ok])) if ok else 0.0)


def poisson_trace(rng, rate_hz: float, duration_s: float, scene: str, make_camera):
    """Arrival times of a Poisson process and one camera per arrival (make_camera(rng))."""
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return out
        out.append((t, scene, make_camera(rng)))
