"""Camera sharding of one scene over ranks (data-parallel training of one partition, Supp. E.1):
every rank holds the same Gaussians, renders its share of a launch's cameras forward and
backward through the library, and one all-reduce (sum) of the FP32 parameter gradients gives
every rank the gradient of the whole launch (the loss is a sum over cameras, Eq. 2 per pixel).

One process per GPU. The exchange is torch.distributed (NCCL between GPUs, gloo on the CPU):
all gradient arrays of a step are views into one flat buffer, so a step makes exactly one
collective call. Nothing here reads another rank's memory directly.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import native


def shard_cameras(sizes: Sequence[int], world: int) -> list[list[int]]:
    """Splits cameras with `sizes` pixels over `world` ranks: largest first to the rank with the
    fewest pixels so far (ties to the lower rank). Returns each rank's camera indices, ascending;
    every camera goes to exactly one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    owned: list[list[int]] = [[] for _ in range(world)]
    for c in sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k)):
        r = min(range(world), key=lambda k: (load[k], k))
        owned[r].append(c)
        load[r] += int(sizes[c])
    return [sorted(o) for o in owned]


class GradBuffer:
    """Parameter gradients of one scene as views into one flat FP32 buffer: means [n,3], scales
    [n,3], quats [n,4], opacities [n], sh [n,K,3] and appearance [C,3,4] for all C cameras of the
    launch (a rank writes the rows of its own cameras; the others stay zero)."""

    def __init__(self, n: int, K: int, n_cams: int, device="cuda"):
        self.n, self.K, self.C = int(n), int(K), int(n_cams)
        shapes = dict(means=(n, 3), scales=(n, 3), quats=(n, 4), opacities=(n,), sh=(n, K, 3),
                      appearance=(n_cams, 3, 4))
        total = sum(int(torch.Size(s).numel()) for s in shapes.values())
        self.flat = torch.zeros(total, dtype=torch.float32, device=device)
        self.views = {}
        off = 0
        for k, s in shapes.items():
            size = int(torch.Size(s).numel())
            self.views[k] = self.flat[off:off + size].view(s)
            off += size

    def __getitem__(self, k):
        return self.views[k]

    def all_reduce(self, group=None):
        """Sums the buffer over the ranks of `group` (one collective call)."""
        import torch.distributed as dist
        dist.all_reduce(self.flat, op=dist.ReduceOp.SUM, group=group)


def local_grads(ctx: native.Context, g: native.Gaussians, cams: Sequence, mine: Sequence[int], d_out: dict,
                opts: native.Options, buf: GradBuffer, appearances: Optional[Sequence] = None, stream=None):
    """Renders cameras `mine` of the launch (forward and backward through the library) with the
    upstream gradients d_out of those cameras (packed like their outputs) and writes their
    parameter gradients into buf (appearance rows at the cameras' launch indices). Returns the
    forward outputs of these cameras."""
    sub = [cams[c] for c in mine]
    apps = None if appearances is None else [appearances[c] for c in mine]
    buf.flat.zero_()
    if not sub:
        return None
    out, st = native.render_forward(ctx, g, sub, opts, appearances=apps, stream=stream)
    grads = dict(means=buf["means"], scales=buf["scales"], quats=buf["quats"], opacities=buf["opacities"],
                 sh=buf["sh"], appearance=torch.empty((len(sub), 3, 4), device=buf.flat.device))
    native.render_backward(ctx, g, sub, st, d_out, opts, appearances=apps, grads=grads, stream=stream)
    idx = torch.tensor(list(mine), dtype=torch.long, device=buf.flat.device)
    buf["appearance"].index_copy_(0, idx, grads["appearance"])
    st.release()
    return out


def sharded_step(ctx: native.Context, g: native.Gaussians, cams: Sequence, d_out_of, opts: native.Options,
                 buf: GradBuffer, rank: int, world: int, appearances: Optional[Sequence] = None, group=None):
    """One camera-sharded training step: this rank's cameras (shard_cameras by pixel count),
    their forward and backward, then one all-reduce of the gradients. d_out_of(mine) gives the
    upstream gradients of this rank's cameras. Returns (mine, this rank's outputs); buf then
    holds the gradient of the whole launch on every rank."""
    mine = shard_cameras([c.width * c.height for c in cams], world)[rank]
    out = local_grads(ctx, g, cams, mine, d_out_of(mine) if mine else None, opts, buf, appearances)
    buf.all_reduce(group)
    return mine, out
