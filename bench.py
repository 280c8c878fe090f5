"""Benchmark: fwd+bwd ms/step and render FPS of the Gaussian rasterizer at 6M Gaussians, 1080p.

Workload ("city6m_1080p"): the seeded synthetic city (1x1 km grid of 100 m blocks, 20 m
streets, 3-6 box buildings per block, heights 10-80 m; 60% of the Gaussians on the ground,
40% on facades; 6,000,000 Gaussians; SH degree 3; FP32) seen by one 1920x1080 camera 150 m
above the ground with a 45-degree pitch. A step is one training pass of the rasterizer:
render_forward (preprocess, binning, per-tile sorts inside the blend, blend) and render_backward
(blend backward beside the gradient zero fill, projection backward) with fixed upstream gradients
on rgb, depth and alpha.
The inputs (1.4 GB of Gaussians) are larger than L2, so no flush is needed between steps.

Prints one JSON line. `value` is the device-timed ms per fwd+bwd step (CUDA events, inputs
resident in HBM); `e2e` repeats the step through the same API with the step's inputs (the
upstream gradients of the outputs) copied in from pinned host memory and its result (the
rendered outputs the loss is computed on) copied out every step, the Gaussians and their
gradients resident as model state is in training (pipelined over two buffer sets;
`serial_value` without overlap); `e2e.full_copy` also copies the Gaussians in and every
parameter gradient out.
`--impl reference` times the FP64 CPU oracle instead (a bounded sample of the same step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "render FPS and fwd+bwd ms/step at 6M Gaussians 1080p; serve p50/p99 latency"

# Algorithmic work per unit: FP32 operations of one (pixel, Gaussian) evaluation in the forward
# blend (the quadratic form, the exponent's argument, alpha, the clamp and tests, the transmittance
# update and the colour and depth sums) and in the backward blend (the same evaluation, the
# transmittance recovered by a division, the remainder update and the ten per-Gaussian sums).
FLOPS_PER_FWD_EVAL = 20.0
FLOPS_PER_BWD_EVAL = 60.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--gaussians", type=int, default=6_000_000)
    p.add_argument("--width", type=int, default=1920)
    p.add_argument("--height", type=int, default=1080)
    p.add_argument("--tile-cull", type=int, default=1)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp16", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-mlp", action="store_true")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the other configurations (street block, 8-camera city, 30M at 4K) and oracle timings")
    p.add_argument("--serve-rate", type=float, default=200.0)
    p.add_argument("--serve-seconds", type=float, default=2.0)
    p.add_argument("--serve-quick", action="store_true",
                   help="serve the bench's own 6M city at 0.3x the serving configuration's sizes with a 2 s "
                        "trace, instead of the configuration at its own sizes (20M/6M/1.5M levels, 30 s trace)")
    p.add_argument("--serve-full-seconds", type=float, default=30.0)
    return p.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region: a sample every
    5 ms once the sampler is running (start() waits for its first sample), each stamped with the
    host time it arrived; mark() brackets the timed region (the host and the GPU move together
    there, each step's forward synchronising once), and only the samples inside it count. When
    the region is shorter than the sampling interval, the nearest sample after it stands in and
    `samples` says 0."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []  # (host time, line)
        self.window = None

    def start(self, ready_timeout=5.0):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "5"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return
        t_end = time.perf_counter() + ready_timeout
        while not self.lines and time.perf_counter() < t_end:
            time.sleep(0.005)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        time.sleep(0.02)  # the sample that follows the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        lines = self.lines
        inside = lines
        if self.window is not None:
            t0, t1 = self.window
            inside = [x for x in lines if t0 <= x[0] <= t1]
            if not inside:
                inside = [x for x in lines if x[0] > t1][:1]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        n_in = 0
        for t, ln in inside:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            if self.window is None or self.window[0] <= t <= self.window[1]:
                n_in += 1
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"], samples=0)
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=n_in)


# CUDA sources each stage's kernels are built from (besides the shared headers): a stored DRAM
# counter stays valid while these files are unchanged.
KERNEL_SOURCES = {
    "blend_fwd": ["blend_fwd.cu", "tile_util.cuh"],
    "blend_bwd": ["blend_bwd.cu", "tile_util.cuh"],
    "tile_scan": ["binning.cu", "tile_util.cuh"],
    "place": ["binning.cu", "tile_util.cuh"],
    "preprocess": ["preprocess_fwd.cuh", "preprocess.cu", "preprocess_rec.cu"],
    "preprocess_bwd": ["preprocess_fwd.cuh", "preprocess.cu"],
}
COMMON_SOURCES = ["gsr_internal.cuh", "scan_util.cuh"]


def sources_sha256(kernel=None):
    """Hash of the CUDA sources of `kernel` (its files and the internal headers; when None, every
    CUDA source and the public header): a stored counter is only valid for it."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2507_23006_gb300", "csrc")
    if kernel is None:
        files = sorted(glob.glob(os.path.join(csrc, "*.cu*"))) + [os.path.join(ROOT, "include", "gsr.h")]
    else:
        files = [os.path.join(csrc, f) for f in sorted(COMMON_SOURCES + KERNEL_SOURCES[kernel])]
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def stored_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu capture
    (profiles/traffic.json), or None when there is none for the kernel's current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    k = rec.get("kernels", {}).get(kernel)
    if rec.get("workload") != workload or k is None or kernel not in KERNEL_SOURCES:
        return None
    if k.get("sources_sha256") != sources_sha256(kernel):
        return None
    return float(k["dram_bytes_per_launch"])


def stored_ncu_us(kernel, workload):
    """The kernel's duration in the committed ncu capture (launched alone, cold), or None when
    there is none for its current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    k = rec.get("kernels", {}).get(kernel)
    if rec.get("workload") != workload or k is None or kernel not in KERNEL_SOURCES:
        return None
    if k.get("sources_sha256") != sources_sha256(kernel):
        return None
    return float(k["ncu_us"])


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def rank_env():
    """(rank, world size, local rank) from the launcher's environment (1 process without one)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def view_azimuth(rank):
    """The work is sharded by camera: rank r renders the city from its own heading (no data is
    exchanged between ranks)."""
    return 90.0 + 45.0 * rank


def max_over_ranks(x, world, device="cpu"):
    """The largest of every rank's x (all ranks call it; a no-op for one process)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_step(ms_max, world):
    """`world` ranks each finish one step within ms_max: the whole job's time per step."""
    return ms_max / world


def workload_name(n, height):
    return f"city{n / 1e6:g}m_{height}p"


def make_workload(n, width, height, rank=0):
    from paper_2507_23006_gb300 import scenes
    scene = scenes.city(2, n)
    cam = scenes.aerial_camera(width, height, altitude=150.0, pitch_deg=45.0, azimuth_deg=view_azimuth(rank))
    return scene, cam


def cpu_reference(scene, cam, tile_cull, seed=0):
    """The FP64 oracle's fwd+bwd of the whole frame (preprocess, binning and compositing of every
    tile, then the backward with random upstream gradients on every pixel), timed as it stands
    on the host's cores."""
    import oracle
    opts = oracle.Opts(tile_cull=bool(tile_cull))
    T = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    up = np.random.default_rng(seed).normal(size=(cam.width * cam.height, 6))
    t0 = time.perf_counter()
    oracle.render(scene, [cam], opts, want_pairs=False)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.backward(scene, [cam], up, opts)
    t_bwd = time.perf_counter() - t0
    return dict(ms_per_step=(t_fwd + t_bwd) * 1e3, sample_s=t_fwd + t_bwd, cores=oracle.num_threads(),
                sample=(f"the whole frame: FP64 preprocess and binning of all {scene.n} Gaussians and "
                        f"compositing of all {T} tiles, forward and backward"))


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    scene, cam = make_workload(args.gaussians, args.width, args.height)
    steps = []
    cores = None
    sample = ""
    for k in range(args.warmup + args.steps):
        r = cpu_reference(scene, cam, args.tile_cull, seed=k)
        cores, sample = r["cores"], r["sample"]
        if k >= args.warmup:
            steps.append(r["ms_per_step"])
    ms = float(np.mean(steps))
    line = dict(metric=METRIC, value=ms, unit="ms/step", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms, higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=dict(workload=workload_name(args.gaussians, args.height), n_gaussians=args.gaussians, width=args.width, height=args.height,
                            tile_cull=bool(args.tile_cull), l2="inputs larger than L2"),
                cpu_baseline=dict(value=ms, unit="ms/step", cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=ms, unit="ms/step", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# FP32 ALU peak: 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# algorithmic flops per visible record of the appearance-transform backward (an FMA is 2):
# recompute 2 (16*32 + 32*4), back through both layers to l_G 2 (4*32 + 32*16), weight-gradient
# outer products of w1's Gaussian part and w2 2 (32*16 + 4*32), bias sums 32 + 4
MLP_BWD_FLOPS_PER_RECORD = 2 * (16 * 32 + 32 * 4) * 3 + 36


def run_mlp_leg(args, ctx, g, cam, opts, d_out, outs, stream, dev, rank):
    """The training step with the per-Gaussian appearance transform (Sec. 3.5.1) on: random
    embeddings and weights, the same Gaussians and camera. Reports the step time, the stages the
    transform touches and the roofline of its backward kernel (ALU-bound, FP32)."""
    import torch
    from paper_2507_23006_gb300 import native

    gen = torch.Generator(device=dev).manual_seed(4321 + rank)
    mlp = native.AppearanceMLP(torch.randn((g.n, 16), device=dev, generator=gen),
                               torch.randn((1, 32), device=dev, generator=gen),
                               0.3 * torch.randn(native.MLP_PARAMS, device=dev, generator=gen))
    gm = native.Gaussians(g.means, g.scales, g.quats, g.opacities, g.sh, 3, None, mlp)
    grads = native.param_grads(ctx, gm, 1)
    out_m = {k: torch.empty_like(v) for k, v in outs.items()}

    def step():
        native.zero_param_grads(ctx, gm, grads)
        _, st = native.render_forward(ctx, gm, [cam], opts, outputs=out_m)
        native.render_backward(ctx, gm, [cam], st, d_out, opts, grads=grads)
        return st

    for _ in range(3):
        st = step()
    torch.cuda.synchronize()
    V = st.info()["n_visible"]
    del st
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st = step()
        del st
    e1.record(stream)
    torch.cuda.synchronize()
    # stage times from a second, profiled pass (events around the three stages only)
    stages = ["preprocess", "appearance_bwd", "preprocess_bwd"]
    ctx.profile(True, False, stages=stages)
    ctx.profile_collect()
    for _ in range(args.steps):
        st = step()
        del st
    torch.cuda.synchronize()
    prof = ctx.profile_collect()
    ctx.profile(False, False)
    stage_ms = {k: prof["ms"][k] / max(prof["launches"][k], 1) for k in stages}
    achieved = MLP_BWD_FLOPS_PER_RECORD * V / (stage_ms["appearance_bwd"] * 1e-3) / 1e12
    return dict(ms_per_step=e0.elapsed_time(e1) / args.steps, n_visible=V,
                stage_ms={k: round(v, 4) for k, v in stage_ms.items()},
                appearance_bwd_roofline=dict(bound="alu", achieved=round(achieved, 2), peak=round(FP32_PEAK_TFLOPS, 1),
                                             unit="TFLOP/s", frac=round(achieved / FP32_PEAK_TFLOPS, 3),
                                             flops_per_record=MLP_BWD_FLOPS_PER_RECORD,
                                             peak_source="152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"))


# Algorithmic work of each stage of one step, each figure derived beside it: bytes that must
# cross HBM, FP32 operations and MUFU operations (ex2, reciprocal) of the blends.
def stage_work(n, V, P, tiles, npix, counts):
    fe, be = counts["fwd_evals"], counts["bwd_evals"]
    return {
        # the per-unit figures of the hot-path scope table: 44 B read per Gaussian, 192 B of SH
        # read and a 48 B record written per visible one
        "preprocess": dict(bytes=44.0 * n + 240.0 * V),
        # binning: the record pass of the preprocess counts the pairs per tile from the records it
        # holds (atomics on the per-tile counters, no extra bytes); the scan reads each tile's
        # count and writes its range and cursor; placing reads the 48 bytes of each record that
        # locate it (position, opacity, depth, conic, rectangle) and writes an 8-byte key per pair
        "tile_scan": dict(bytes=16.0 * tiles),
        "place": dict(bytes=48.0 * V + 8.0 * P),
        # the forward blend sorts each tile's keys (lists of at most 1024 pairs; longer ones, none on
        # these workloads, are sorted by a launch of their own): it reads the 8-byte key and writes
        # the 4-byte record index per pair, then reads each pair's 48-byte record
        "blend_fwd": dict(bytes=60.0 * P + 28.0 * npix, flops=FLOPS_PER_FWD_EVAL * fe, mufu=1.0 * fe),
        "blend_bwd": dict(bytes=48.0 * P + 28.0 * npix + 40.0 * V, flops=FLOPS_PER_BWD_EVAL * be, mufu=2.0 * be),
        # the projection backward with the gradient rows: 84 B read and the 44 B non-SH gradient
        # rows written per Gaussian, plus 232 B of SH rows read and written per visible Gaussian
        # (one record per visible Gaussian with one camera)
        "preprocess_bwd": dict(bytes=128.0 * n + 232.0 * V),
        # the zeros the dense-overwrite contract puts in the SH rows of Gaussians without a record
        # (192 B each, side stream, beside the backward blend): reported, not counted in the step
        "gradient_fill": dict(bytes=192.0 * max(n - V, 0), counted=False),
    }


def stage_rooflines(stage_ms, n, V, P, tiles, npix, counts, fp32_tflops, mufu_per_s, hbm_gbs, step_ms):
    """Per stage: the algorithmic time (the largest of bytes / HBM peak, FP32 ops / FP32 peak and
    MUFU ops / MUFU peak) against the measured time; for the step, the sum of the stages'
    algorithmic times (the gradient fill's included) against the step time."""
    out = {}
    total = 0.0
    for k, w in stage_work(n, V, P, tiles, npix, counts).items():
        t = {"hbm": w.get("bytes", 0.0) / (hbm_gbs * 1e9), "alu": w.get("flops", 0.0) / (fp32_tflops * 1e12),
             "mufu": w.get("mufu", 0.0) / mufu_per_s}
        bound = max(t, key=t.get)
        algo_us = t[bound] * 1e6
        if w.get("counted", True):
            total += algo_us
        meas = stage_ms.get(k)
        row = dict(bound=bound, algorithmic_us=round(algo_us, 2))
        if meas:
            row.update(measured_us=round(meas * 1e3, 2), frac=round(algo_us / (meas * 1e3), 3))
        else:
            row.update(measured_us=None, frac=None, note="runs beside the other stages")
        if not w.get("counted", True):
            row["note"] = "zeros forced by the dense-overwrite contract; not counted in the step's algorithmic time"
        out[k] = row
    return out, dict(algorithmic_us=round(total, 1), step_us=round(step_ms * 1e3, 1),
                     frac=round(total / (step_ms * 1e3), 3))


def run_e2e(args, ctx, g, cam, opts, d_out, grads, outs, stream, world, dev, barrier, full_copy=False):
    """The step through the same API with host copies every step, pipelined the way a training
    loop would run it: two sets of device buffers, the copies in and the copies out on their own
    streams, so step i's copy out and step i+1's copy in overlap step i's compute (the link
    carries both directions at once); also the same steps one after another on one stream
    (`serial_value`). By default the step's inputs are the upstream gradients of the outputs (the
    loss's gradient, computed elsewhere) copied in and its result the rendered outputs copied
    out (what the loss is computed on); the Gaussians and their gradients stay on the device, as
    model state does in training. full_copy: the Gaussians are copied in and every parameter
    gradient copied out as well."""
    import torch
    from paper_2507_23006_gb300 import native

    keys = ("means", "scales", "quats", "opacities", "sh")
    host = {k: getattr(g, k).to("cpu").pin_memory() for k in keys} if full_copy else {}
    host_up = {k: v.to("cpu").pin_memory() for k, v in d_out.items()}
    gkeys = [k for k, v in grads.items() if v is not None] if full_copy else []
    okeys = list(outs)
    h2d = sum(v.numel() * v.element_size() for v in host.values()) + \
        sum(v.numel() * v.element_size() for v in host_up.values())
    d2h = sum(grads[k].numel() * grads[k].element_size() for k in gkeys) + \
        sum(outs[k].numel() * outs[k].element_size() for k in okeys)
    # buffer set 0 is the bench's own; set 1 a copy
    gs = [g, native.Gaussians(*(getattr(g, k).clone() for k in keys), 3) if full_copy else g]
    ds = [d_out, {k: v.clone() for k, v in d_out.items()}]
    grs = [grads, {k: (torch.empty_like(v) if v is not None else None) for k, v in grads.items()}]
    os_ = [outs, {k: torch.empty_like(v) for k, v in outs.items()}]
    hgs = [{k: torch.empty(grads[k].shape, dtype=grads[k].dtype, pin_memory=True) for k in gkeys} for _ in range(2)]
    hos = [{k: torch.empty(outs[k].shape, dtype=outs[k].dtype, pin_memory=True) for k in okeys} for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def copy_in(b):
        for k in host:
            getattr(gs[b], k).copy_(host[k], non_blocking=True)
        for k, v in host_up.items():
            ds[b][k].copy_(v, non_blocking=True)

    def compute(b):
        native.zero_param_grads(ctx, gs[b], grs[b])
        _, st = native.render_forward(ctx, gs[b], [cam], opts, outputs=os_[b])
        native.render_backward(ctx, gs[b], [cam], st, ds[b], opts, grads=grs[b])

    def copy_out(b):
        for k in gkeys:
            hgs[b][k].copy_(grs[b][k], non_blocking=True)
        for k in okeys:
            hos[b][k].copy_(os_[b][k], non_blocking=True)

    def pipelined_step(i):
        b = i % 2
        s_in.wait_event(ev_comp[b])  # step i-2 has finished reading this set's inputs
        with torch.cuda.stream(s_in):
            copy_in(b)
            ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        stream.wait_event(ev_out[b])  # step i-2's results have left this set
        compute(b)
        ev_comp[b].record(stream)
        s_out.wait_event(ev_comp[b])
        with torch.cuda.stream(s_out):
            copy_out(b)
            ev_out[b].record(s_out)

    def timed(fn):
        torch.cuda.synchronize()
        barrier()
        x0 = torch.cuda.Event(enable_timing=True)
        x1 = torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        s_in.wait_event(x0)
        s_out.wait_event(x0)
        for i in range(args.steps):
            fn(i)
        for e in ev_out:
            stream.wait_event(e)
        x1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(x0.elapsed_time(x1) / args.steps, world, dev)

    def serial_step(i):
        copy_in(0)
        compute(0)
        copy_out(0)

    for i in range(4):
        pipelined_step(i)
    torch.cuda.synchronize()
    pipe_ms = timed(pipelined_step)
    serial_ms = timed(serial_step)
    what = ("Gaussians and upstream gradients in, parameter gradients and outputs out" if full_copy else
            "upstream gradients in, rendered outputs out; Gaussians and gradients resident")
    return dict(value=job_ms_per_step(pipe_ms, world), unit="ms/step", h2d_bytes_per_step=int(h2d),
                d2h_bytes_per_step=int(d2h), copies=what,
                mode="pipelined: 2 buffer sets, copies in and out on their own streams",
                serial_value=job_ms_per_step(serial_ms, world),
                link_gbs=round((h2d + d2h) / (pipe_ms * 1e-3) / 1e9, 1))


def _events_ms(fn, k, stream):
    """Mean device milliseconds of fn() over k calls (CUDA events on `stream`, after 2 untimed)."""
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def _upstream_t(npix, dev, seed):
    import torch
    gen = torch.Generator(device=dev).manual_seed(seed)
    return dict(rgb=torch.randn((npix, 3), device=dev, generator=gen),
                depth_acc=torch.randn(npix, device=dev, generator=gen) * 1e-2,
                alpha=torch.randn(npix, device=dev, generator=gen))


def run_configs(args, ctx, dev, stream):
    """The other configurations of the hot path, on the device with inputs resident (CUDA events,
    2 untimed calls first): the 500k street block at 1080p with a per-image 3x4 transform (forward
    and backward timed apart); the 6M city seen by 8 cameras of mixed resolution in one launch,
    FP32 and FP16 SH side by side, with the image error of each against the FP64 oracle on the
    original FP32 inputs (camera 0, every pixel); the 30M street-level scene at 3840x2160 with FP16
    SH in recompute mode (step time and peak device memory)."""
    import torch
    import oracle
    from paper_2507_23006_gb300 import native, scenes
    k = max(3, min(args.steps, 10))
    out = {}
    # street block (500k, 1080p)
    sc, cam = scenes.street_block(1, 500_000), scenes.street_block_camera()
    rng = np.random.default_rng(1)
    aff = np.concatenate([np.eye(3), np.zeros((3, 1))], 1) + rng.normal(0, 0.01, (3, 4))
    aff_t = torch.tensor(aff, dtype=torch.float32, device=dev)
    g = native.Gaussians.from_scene(sc, device=dev)
    opts = native.Options(tile_cull=True)
    npix = cam.width * cam.height
    up = _upstream_t(npix, dev, 5)
    grads = native.param_grads(ctx, g, 1)
    holder = {}

    def fwd():
        holder["st"] = native.render_forward(ctx, g, [cam], opts, appearances=[aff_t])[1]

    def bwd():
        native.render_backward(ctx, g, [cam], holder["st"], up, opts, appearances=[aff_t], grads=grads)

    fms = _events_ms(fwd, k, stream)
    bms = _events_ms(bwd, k, stream)
    info = holder["st"].info()
    out["street_block_500k_1080p"] = dict(fwd_ms=round(fms, 4), bwd_ms=round(bms, 4), visible=info["n_visible"],
                                          pairs=info["n_pairs"], appearance_affine=True)
    del holder["st"], g, grads
    # city, 8 cameras of mixed resolution in one launch
    sc = scenes.city(2, 6_000_000)
    cams = scenes.city_batch_cameras(2)
    npix = sum(c.width * c.height for c in cams)
    up = _upstream_t(npix, dev, 6)
    city = {}
    renders = {}
    for name, shd in (("fp32", torch.float32), ("fp16_sh", torch.float16)):
        g = native.Gaussians.from_scene(sc, device=dev, sh_dtype=shd)
        grads = native.param_grads(ctx, g, len(cams))

        def step():
            native.zero_param_grads(ctx, g, grads)
            _, st = native.render_forward(ctx, g, cams, opts)
            native.render_backward(ctx, g, cams, st, up, opts, grads=grads)

        ms = _events_ms(step, k, stream)
        o, st = native.render_forward(ctx, g, cams, opts)
        torch.cuda.synchronize()
        renders[name] = {kk: v[: cams[0].width * cams[0].height].double().cpu().numpy() for kk, v in o.items()}
        city[name] = dict(ms_per_launch=round(ms, 4), visible=st.info()["n_visible"], pairs=st.info()["n_pairs"],
                          sh_bytes_per_gaussian=48 * (4 if shd == torch.float32 else 2))
        del g, grads, st, o
    ref = oracle.render(sc, [cams[0]], oracle.Opts(tile_cull=True), want_pairs=False)
    um = ref.mark == 0
    for name, r in renders.items():
        city[name]["vs_oracle_cam0"] = dict(
            rgb_max_abs=float(np.abs(r["rgb"][um] - ref.img[um, 0:3]).max()),
            alpha_max_abs=float(np.abs(r["alpha"][um] - ref.img[um, 5]).max()),
            depth_acc_max_rel=float((np.abs(r["depth_acc"][um] - ref.img[um, 3]) /
                                     np.maximum(ref.img[um, 3], 1e-9)).max()),
            pixels=int(um.sum()), marked=int((~um).sum()))
    out["city6m_8cam_mixed"] = dict(cameras=[f"{c.width}x{c.height}" for c in cams], **city)
    # 30M street-level at 4K, FP16 SH, recompute mode
    sc = scenes.large_scene(4, 30_000_000)
    cam = scenes.street_level_camera(3840, 2160)
    g = native.Gaussians.from_scene(sc, device=dev, sh_dtype=torch.float16)
    del sc
    ropts = native.Options(tile_cull=True, save_state=False)
    up = _upstream_t(cam.width * cam.height, dev, 7)
    grads = native.param_grads(ctx, g, 1)

    def step4():
        native.zero_param_grads(ctx, g, grads)
        _, st = native.render_forward(ctx, g, [cam], ropts)
        native.render_backward(ctx, g, [cam], st, up, ropts, grads=grads)

    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    ms = _events_ms(step4, max(3, k // 2), stream)
    peak = torch.cuda.max_memory_allocated() + ctx.workspace_bytes()
    _, st = native.render_forward(ctx, g, [cam], ropts)
    out["large30m_4k_recompute_fp16sh"] = dict(ms_per_step=round(ms, 3), peak_device_gib=round(peak / 2 ** 30, 2),
                                                visible=st.info()["n_visible"], pairs=st.info()["n_pairs"])
    del g, grads, st
    torch.cuda.empty_cache()
    return out


def oracle_timings():
    """The FP64 oracle as it stands, forward and backward of the whole frame: the 10k box scene
    (256x256) and the 500k street block (1080p) with every host core and with one, the 6M city's
    first 8-camera-launch camera (1600x1067) with every core. (The headline frame is cpu_baseline.)"""
    import oracle
    from paper_2507_23006_gb300 import scenes
    full = oracle.num_threads()
    out = {"cores": full}
    cases = [("box10k_256", scenes.box_scene(0, 10_000), scenes.box_camera(), (full, 1)),
             ("street_block500k_1080p", scenes.street_block(1, 500_000), scenes.street_block_camera(), (full, 1)),
             ("city6m_1600x1067_cam0", scenes.city(2, 6_000_000), scenes.city_batch_cameras(2)[0], (full,))]
    try:
        for name, sc, cam, threads in cases:
            row = {}
            for t in threads:
                oracle.set_num_threads(t)
                r = cpu_reference(sc, cam, True)
                row[f"{t}_cores_ms"] = round(r["ms_per_step"], 1)
            out[name] = row
    finally:
        oracle.set_num_threads(full)
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2507_23006_gb300 import native

    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    scene, cam = make_workload(args.gaussians, args.width, args.height, rank)
    ctx = native.Context(local_rank)
    g = native.Gaussians.from_scene(scene, device=dev)
    opts = native.Options(tile_cull=bool(args.tile_cull), save_state=True)
    npix = cam.width * cam.height
    gen = torch.Generator(device=dev).manual_seed(1234 + rank)
    d_out = dict(rgb=torch.randn((npix, 3), device=dev, generator=gen),
                 depth_acc=torch.randn(npix, device=dev, generator=gen) * 1e-2,
                 alpha=torch.randn(npix, device=dev, generator=gen))
    outs = dict(rgb=torch.empty((npix, 3), device=dev), depth_acc=torch.empty(npix, device=dev),
                depth_exp=torch.empty(npix, device=dev), alpha=torch.empty(npix, device=dev))
    n = g.n
    K = int(g.sh.shape[1])
    grads = dict(means=torch.empty((n, 3), device=dev), scales=torch.empty((n, 3), device=dev),
                 quats=torch.empty((n, 4), device=dev), opacities=torch.empty(n, device=dev),
                 sh=torch.empty((n, K, 3), device=dev), appearance=torch.empty((1, 3, 4), device=dev),
                 absgrad=None)

    def step():
        # the gradient arrays are zeroed beside the backward blend (gsr_param_grads_zero)
        native.zero_param_grads(ctx, g, grads)
        _, st = native.render_forward(ctx, g, [cam], opts, outputs=outs)
        native.render_backward(ctx, g, [cam], st, d_out, opts, grads=grads)
        return st

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        st = step()
    torch.cuda.synchronize()
    info = st.info()
    del st
    stream = torch.cuda.current_stream()
    # per-stage device times from an untimed pass with events around every stage (they add a
    # little idle time between stages); it also names the dominant kernel
    ctx.profile(True, False)
    ctx.profile_collect()
    for _ in range(args.steps):
        st = step()
        del st
    torch.cuda.synchronize()
    prof = ctx.profile_collect()
    dom = max((k for k in native.STAGES if k != "between_stages"), key=prof["ms"].get)
    # the timed loop records events around the dominant kernel only (its roofline duration)
    ctx.profile(True, False, stages=[dom])
    ctx.profile_collect()
    sampler = ClockSampler(local_rank)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_host0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        st = step()
        del st
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(t_host0, time.perf_counter())
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    timed = ctx.profile_collect()
    ctx.profile(False, False)
    dom_ms = timed["ms"][dom] / max(timed["launches"][dom], 1)
    ms = max_over_ranks(ms, world, dev)
    # forward-only frames per second (render path without state)
    for _ in range(2):
        native.render_forward(ctx, g, [cam], opts, outputs=outs, want_state=False)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        native.render_forward(ctx, g, [cam], opts, outputs=outs, want_state=False)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = max_over_ranks(f0.elapsed_time(f1) / args.steps, world, dev)
    # blend evaluation counts (deterministic; one counting pass outside the timed region)
    ctx.profile(True, True)
    st = step()
    torch.cuda.synchronize()
    counts = ctx.profile_collect()["counters"]
    ctx.profile(False, False)
    del st

    # the same step with FP16 attribute and SH storage (FP32 projection, blending, gradients)
    fp16 = None
    if not args.no_fp16:
        import torch as _t
        g16 = native.Gaussians(g.means, g.scales.half(), g.quats.half(), g.opacities.half(), g.sh.half(), 3)
        out16 = {k: _t.empty_like(v) for k, v in outs.items()}

        def step16():
            native.zero_param_grads(ctx, g16, grads)
            _, st16 = native.render_forward(ctx, g16, [cam], opts, outputs=out16)
            native.render_backward(ctx, g16, [cam], st16, d_out, opts, grads=grads)

        for _ in range(2):
            step16()
        native.render_forward(ctx, g, [cam], opts, outputs=outs, want_state=False)
        torch.cuda.synchronize()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(args.steps):
            step16()
        h1.record(stream)
        torch.cuda.synchronize()
        native.render_forward(ctx, g16, [cam], opts, outputs=out16, want_state=False)
        torch.cuda.synchronize()
        fp16 = dict(ms_per_step=h0.elapsed_time(h1) / args.steps,
                    rgb_max_abs_vs_fp32=float((out16["rgb"] - outs["rgb"]).abs().max()),
                    rgb_mean_abs_vs_fp32=float((out16["rgb"] - outs["rgb"]).abs().mean()),
                    bytes_per_gaussian=int(12 + 2 * (3 + 4 + 1) + 2 * 48))

    # the same step with the pairs ordered by global onesweep radix sorts instead of per-tile sorts
    # (same results): step time and binning stage times of both
    binning = None
    if not args.no_configs:
        binning = {}
        bstages = ["tile_count", "tile_scan", "readback", "place", "tile_sort", "depth_sort", "ranges"]
        for name, glob in (("per_tile_sort", False), ("global_onesweep", True)):
            o2 = native.Options(tile_cull=bool(args.tile_cull), save_state=True, global_sort=glob)

            def step_b():
                native.zero_param_grads(ctx, g, grads)
                _, stb = native.render_forward(ctx, g, [cam], o2, outputs=outs)
                native.render_backward(ctx, g, [cam], stb, d_out, o2, grads=grads)

            ms_b = _events_ms(step_b, max(3, min(args.steps, 10)), stream)
            ctx.profile(True, False)
            ctx.profile_collect()
            for _ in range(5):
                step_b()
            torch.cuda.synchronize()
            pr = ctx.profile_collect()
            ctx.profile(False, False)
            binning[name] = dict(ms_per_step=round(ms_b, 4),
                                 stage_us={k: round(pr["ms"][k] / 5 * 1e3, 1) for k in bstages if pr["ms"][k] > 0})

    mlp_leg = None if args.no_mlp else run_mlp_leg(args, ctx, g, cam, opts, d_out, outs, stream, dev, rank)

    # end to end through the same API: Gaussians from pinned host memory in, gradients out
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, ctx, g, cam, opts, d_out, grads, outs, stream, world, dev, barrier)
        e2e["full_copy"] = run_e2e(args, ctx, g, cam, opts, d_out, grads, outs, stream, world, dev, barrier,
                                   full_copy=True)

    configs = None if args.no_configs or rank != 0 else run_configs(args, ctx, dev, stream)

    serve_stats = None
    if not args.no_serve and args.serve_quick:
        serve_stats = run_serve(scene, args)
    serve_full = run_serve_full(args) if not args.no_serve and not args.serve_quick and rank == 0 else None

    if rank != 0:
        return 0
    # roofline of the dominant kernel
    stage_ms = {k: v / max(args.steps, 1) for k, v in prof["ms"].items()}
    launches = {k: v / max(args.steps, 1) for k, v in prof["launches"].items()}
    sm_mhz = clocks.get("sm_mhz") or 1455.0
    props = torch.cuda.get_device_properties(local_rank)
    sms = props.multi_processor_count
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s at the sampled SM clock
    hbm, hbm_kind = peaks()
    V, P = info["n_visible"], info["n_pairs"]
    if dom in ("blend_fwd", "blend_bwd"):
        evals = counts["fwd_evals"] if dom == "blend_fwd" else counts["bwd_evals"]
        flops = evals * (FLOPS_PER_FWD_EVAL if dom == "blend_fwd" else FLOPS_PER_BWD_EVAL)
        achieved = flops / (dom_ms * 1e-3) / 1e12
        roof = dict(kernel=dom, launch_ms=dom_ms, bound="alu", achieved=achieved, peak=fp32_peak, unit="TFLOP/s",
                    frac=achieved / fp32_peak, traffic=stored_traffic(dom, workload_name(n, cam.height)),
                    peak_source=f"{sms} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (sampled)")
        alone_us = stored_ncu_us(dom, workload_name(n, cam.height))
        if dom == "blend_bwd" and alone_us:
            # live, the gradient zero fill runs beside this kernel; the same launch alone (ncu,
            # cold, no fill beside it) for comparison
            roof["alone_ms_ncu"] = alone_us * 1e-3
            roof["frac_alone_ncu"] = flops / (alone_us * 1e-6) / 1e12 / fp32_peak
    else:
        work = stage_work(n, V, P, info["n_tiles"], cam.width * cam.height, counts)
        per_unit = {k: w.get("bytes", 0.0) for k, w in work.items()}
        bytes_ = per_unit.get(dom, 0.0)
        achieved = bytes_ / (dom_ms * 1e-3) / 1e9
        roof = dict(kernel=dom, launch_ms=dom_ms, bound="hbm", achieved=achieved, peak=hbm, unit="GB/s", frac=achieved / hbm,
                    traffic=stored_traffic(dom, workload_name(n, cam.height)),
                    peak_source=f"{hbm_kind} HBM copy bandwidth")
    stage_roof, step_roof = stage_rooflines(stage_ms, n, V, P, info["n_tiles"], cam.width * cam.height, counts,
                                            fp32_peak, sms * 16 * sm_mhz * 1e6, hbm, ms)
    cpu = None
    if not args.no_cpu_baseline:
        r = cpu_reference(scene, cam, args.tile_cull)
        cpu = dict(value=r["ms_per_step"], unit="ms/step", cores=r["cores"], kind="oracle", sample=r["sample"],
                   sample_seconds=round(r["sample_s"], 1))
        if not args.no_configs:
            cpu["other_configs"] = oracle_timings()
    value = job_ms_per_step(ms, world)
    line = dict(metric=METRIC, value=value, unit="ms/step", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms, higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f32",
                data="synthetic",
                config=dict(workload=workload_name(n, cam.height), n_gaussians=n, width=cam.width, height=cam.height,
                            tile_cull=bool(args.tile_cull), sh_degree=3, attributes="f32",
                            l2="inputs larger than L2 (1.4 GB), no flush", parallelism=f"replicas{world}"),
                render_fps=1000.0 / fwd_ms * world, fwd_ms=fwd_ms,
                # weak scaling: every rank renders its own view; the rank step time (max over ranks)
                # and the views the whole job trains per second, apart from `value`
                per_rank_ms_per_step=ms, views_per_s=world * 1000.0 / ms,
                stages_ms=stage_ms, visible=V, pairs=P, max_tile_pairs=info.get("max_tile_pairs"), counters=counts,
                roofline=roof, stage_roofline=stage_roof, step_roofline=step_roof,
                cpu_baseline=cpu, e2e=e2e, clocks=clocks, fp16_storage=fp16, appearance_mlp=mlp_leg, serve=serve_stats,
                configs=configs, binning=binning)
    if serve_full is not None:
        line["serve"] = serve_full  # the serving configuration at its own sizes
    line["gpu_launches"] = int(args.steps * kernels_per_step(args.tile_cull, info))
    print(json.dumps(line), flush=True)
    return 0


def _serve_cameras():
    from paper_2507_23006_gb300 import scenes
    res_choices = [(1280, 720), (1920, 1080), (3840, 2160)]

    def make_cam(rng):
        w, h = res_choices[int(rng.integers(0, 3))]
        if rng.uniform() < 0.5:
            return scenes.walkthrough_camera(rng, w, h)
        return scenes.aerial_camera(w, h, altitude=rng.uniform(80, 300), pitch_deg=rng.uniform(30, 89),
                                    target=(rng.uniform(-500, 500), rng.uniform(-500, 500), 0.0),
                                    azimuth_deg=rng.uniform(0, 360))
    return make_cam


def _serve_pair(levels, full, budget, rate, seconds, warm_s):
    """The FP16 LOD server and the plain FP32 full-detail renderer on the same Poisson trace
    (after a warm-up trace), then a burst of 200 simultaneous requests (saturated frames/s)."""
    import torch
    from paper_2507_23006_gb300 import serve
    make_cam = _serve_cameras()
    out = {}
    for name, lodscene, dt, gb in (("lod_fp16", levels, torch.float16, budget), ("full_fp32", full, torch.float32, 0)):
        srv = serve.RenderServer(slots=4, gaussian_budget=gb, keep_results=False)
        srv.add_scene("city", lodscene, attr_dtype=dt, sh_dtype=dt)
        srv.run_trace(serve.poisson_trace(np.random.default_rng(7), rate, warm_s, "city", make_cam))
        st = srv.run_trace(serve.poisson_trace(np.random.default_rng(8), rate, seconds, "city", make_cam))
        rng = np.random.default_rng(9)
        burst = srv.run_trace([(0.0, "city", make_cam(rng)) for _ in range(200)])
        srv.close()
        out[name] = {k: st[k] for k in ("p50_ms", "p99_ms", "mean_ms", "fps", "served", "failed", "max_in_flight",
                                        "mean_batch", "mean_selected")}
        out[name]["saturated_fps"] = burst["fps"]
        out[name]["saturated_mean_batch"] = burst["mean_batch"]  # views per launch under the burst
        out[name]["saturated_p99_ms"] = burst["p99_ms"]
        errs = sorted({r.error for r in st["requests"] + burst["requests"] if r.error})
        if errs:
            out[name]["errors"] = errs[:3]
        del srv
        torch.cuda.empty_cache()
    return out


def _serve_psnr(levels, full, budget, views=12):
    """PSNR of the FP16-attribute render of each view's selected LOD set against the FP32 render
    of the same set (the bar), and against the full-detail FP32 render (for information)."""
    import torch
    from paper_2507_23006_gb300 import native, serve
    make_cam = _serve_cameras()
    ctx = native.Context(0)
    g32 = native.Gaussians.from_scene(levels.gaussians)
    g16 = native.Gaussians.from_scene(levels.gaussians, attr_dtype=torch.float16, sh_dtype=torch.float16)
    gf = native.Gaussians.from_scene(full.gaussians)
    sel = serve.RenderServer(slots=1, gaussian_budget=budget)
    sel.add_scene("city", levels)
    opts = native.Options(tile_cull=True)
    rng = np.random.default_rng(11)
    same, vs_full = [], []

    def psnr(a, b):
        mse = float(((a.clamp(0, 1) - b.clamp(0, 1)) ** 2).mean())
        return 10.0 * math.log10(1.0 / max(mse, 1e-20))
    for _ in range(views):
        cam = make_cam(rng)
        segs, _, _ = sel.select("city", cam)
        r32, _ = native.render_forward(ctx, native.Gaussians(g32.means, g32.scales, g32.quats, g32.opacities, g32.sh, 3,
                                                             segs), [cam], opts, want_state=False)
        r16, _ = native.render_forward(ctx, native.Gaussians(g16.means, g16.scales, g16.quats, g16.opacities, g16.sh, 3,
                                                             segs), [cam], opts, want_state=False)
        rf, _ = native.render_forward(ctx, gf, [cam], opts, want_state=False)
        same.append(psnr(r16["rgb"], r32["rgb"]))
        vs_full.append(psnr(r16["rgb"], rf["rgb"]))
    sel.close()
    ctx.close()
    return dict(min_psnr_fp16_vs_fp32_same_set_db=round(min(same), 2),
                mean_psnr_lod_fp16_vs_full_fp32_db=round(float(np.mean(vs_full)), 2), views=views)


def run_serve(scene, args):
    """Serving on the bench's city: detail levels (the 6M scene and two merged coarser levels,
    0.3x the 20M / 6M / 1.5M of the reference configuration, budget scaled alike), Poisson
    arrivals, resolutions drawn from 720p / 1080p / 4K, half walk-through and half aerial poses.
    The FP16 LOD server and the plain FP32 full-detail renderer serve the same trace."""
    from paper_2507_23006_gb300 import lod
    t0 = time.perf_counter()
    mid = lod.merge_to_count(scene, int(0.3 * scene.n))
    coarse = lod.merge_to_count(mid, int(0.075 * scene.n))
    levels = lod.build_lod([coarse, mid, scene])
    full = lod.build_lod([scene])
    build_s = time.perf_counter() - t0
    budget = int(4_000_000 * scene.n / 20_000_000)
    out = _serve_pair(levels, full, budget, args.serve_rate, args.serve_seconds, 0.5)
    out["config"] = dict(levels=levels.level_sizes, partitions=int(levels.aabb.shape[0]), gaussian_budget=budget,
                         thresholds_m=[100.0, 200.0], rate_hz=args.serve_rate, seconds=args.serve_seconds,
                         resolutions=["1280x720", "1920x1080", "3840x2160"], slots=4, lod_build_s=round(build_s, 1))
    return out


def run_serve_full(args):
    """The serving configuration at its own sizes: a 20M-Gaussian city (seed 3) merged to 6M
    and 1.5M levels over 100 m partitions, a 4M-Gaussian budget, Poisson arrivals at 200 req/s
    for 30 s after a 2 s warm-up, 720p / 1080p / 4K, half walk-through and half aerial poses."""
    from paper_2507_23006_gb300 import lod, scenes
    t0 = time.perf_counter()
    fine = scenes.city(3, 20_000_000)
    mid = lod.merge_to_count(fine, 6_000_000)
    coarse = lod.merge_to_count(mid, 1_500_000)
    levels = lod.build_lod([coarse, mid, fine])
    full = lod.build_lod([fine])
    build_s = time.perf_counter() - t0
    budget = 4_000_000
    out = _serve_pair(levels, full, budget, args.serve_rate, args.serve_full_seconds, 2.0)
    out["psnr"] = _serve_psnr(levels, full, budget)
    out["config"] = dict(levels=levels.level_sizes, partitions=int(levels.aabb.shape[0]), gaussian_budget=budget,
                         thresholds_m=[100.0, 200.0], rate_hz=args.serve_rate, seconds=args.serve_full_seconds,
                         warmup_s=2.0, resolutions=["1280x720", "1920x1080", "3840x2160"], slots=4,
                         lod_build_s=round(build_s, 1))
    return out


def kernels_per_step(tile_cull, info):
    """Kernels of ours launched per fwd+bwd step (memsets excluded)."""
    k = 2                      # preprocess: cull pass, record pass (which counts the pairs per tile)
    k += 1                     # tile scan
    k += 1 if int(info["n_pairs"]) > 0 else 0    # pair placement
    k += 1 if int(info.get("max_tile_pairs", 0)) > 1024 else 0  # sort of the lists over 1024 pairs
    k += 1                     # blend forward (sorts the other lists)
    k += 1                     # gradient zero fill (side stream)
    k += 1 + 1                 # blend backward, preprocess backward
    return k


def main():
    args = parse()
    rank, world, local_rank = rank_env()
    if world > 1:
        import torch.distributed as dist
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
