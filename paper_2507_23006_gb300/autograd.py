"""torch.autograd wrapper around render_forward / render_backward.

`rasterize` takes unconstrained training parameters (log-scales, opacity logits, raw
quaternions, SH coefficients, optional per-image 3x4 appearance transforms, optional per-Gaussian
appearance transform of Sec. 3.5.1: Gaussian and image embeddings and its packed weights), applies the
activations in torch (exp, sigmoid), and renders through the CUDA library; backward calls the
library's backward and lets torch chain the activations. With ``recompute=True`` the forward
keeps only 16 bytes per pixel and the backward re-runs the binning (Sec. 3.1 rendering of
tens of millions of Gaussians at 4K without storing the pair lists).
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import native


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(fctx, means, scales, quats, opacities, sh, appearance, gauss_embed, image_embed, mlp_params, lib_ctx,
                cams, opts, sh_degree, segments):
        mlp = None
        if gauss_embed is not None:
            mlp = native.AppearanceMLP(gauss_embed.contiguous().float(), image_embed.contiguous().float(),
                                       mlp_params.contiguous().float())
        g = native.Gaussians(means.contiguous(), scales.contiguous(), quats.contiguous(), opacities.contiguous(),
                             sh.contiguous(), sh_degree, segments, mlp)
        apps = None
        if appearance is not None:
            appearance = appearance.contiguous()
            apps = [appearance[c] for c in range(len(cams))]
        grads = None
        if any(fctx.needs_input_grad[:9]):
            # the gradient arrays to zero (the backward queues the fill beside its blend)
            grads = native.param_grads(lib_ctx, g, len(cams), opts.absgrad)
            native.zero_param_grads(lib_ctx, g, grads)
        outs, state = native.render_forward(lib_ctx, g, cams, opts, appearances=apps)
        fctx.grads = grads
        fctx.state = state
        fctx.lib_ctx = lib_ctx
        fctx.cams = cams
        fctx.opts = opts
        fctx.g = g
        fctx.apps = apps
        fctx.has_app = appearance is not None
        fctx.attr_dtype = scales.dtype
        fctx.sh_dtype = sh.dtype
        return outs["rgb"], outs["depth_acc"], outs["depth_exp"], outs["alpha"]

    @staticmethod
    def backward(fctx, d_rgb, d_dacc, d_dexp, d_alpha):
        def c(t):
            return None if t is None else t.contiguous().float()
        grads = native.render_backward(fctx.lib_ctx, fctx.g, fctx.cams, fctx.state,
                                       dict(rgb=c(d_rgb), depth_acc=c(d_dacc), depth_exp=c(d_dexp),
                                            alpha=c(d_alpha)), fctx.opts, appearances=fctx.apps, grads=fctx.grads)
        fctx.state.release()
        fctx.state = None
        fctx.grads = None
        app = grads["appearance"] if fctx.has_app else None
        m = fctx.g.mlp is not None
        return (grads["means"], grads["scales"].to(fctx.attr_dtype), grads["quats"].to(fctx.attr_dtype),
                grads["opacities"].to(fctx.attr_dtype), grads["sh"].to(fctx.sh_dtype), app,
                grads["gauss_embed"] if m else None, grads["image_embed"] if m else None,
                grads["mlp_params"] if m else None, None, None, None, None, None)


def rasterize(lib_ctx: native.Context, means: torch.Tensor, log_scales: torch.Tensor, quats: torch.Tensor,
              opacity_logits: torch.Tensor, sh: torch.Tensor, cams: Sequence, appearance: Optional[torch.Tensor] = None,
              sh_degree: int = 3, opts: Optional[native.Options] = None, recompute: bool = False,
              segments=None, attr_dtype: Optional[torch.dtype] = None, gauss_embed: Optional[torch.Tensor] = None,
              image_embed: Optional[torch.Tensor] = None, mlp_params: Optional[torch.Tensor] = None):
    """Differentiable render of the cameras (packed). Returns rgb [P,3], depth_acc [P],
    depth_exp [P], alpha [P]. Activations: scale = exp(log_scale), opacity = sigmoid(logit).
    attr_dtype (f16 / bf16) stores the activated attributes in that precision; projection,
    blending and gradients stay FP32. gauss_embed [n,16], image_embed [len(cams),32] and
    mlp_params [1700] (w1 | b1 | w2 | b2) switch on the per-Gaussian appearance transform."""
    opts = opts or native.Options()
    opts = native.Options(eps2d=opts.eps2d, antialiased=opts.antialiased, tile_cull=opts.tile_cull, bg=opts.bg,
                          save_state=not recompute, absgrad=opts.absgrad)
    scales = torch.exp(log_scales)
    opac = torch.sigmoid(opacity_logits)
    if attr_dtype is not None:
        scales, quats, opac = scales.to(attr_dtype), quats.to(attr_dtype), opac.to(attr_dtype)
    if (gauss_embed is None) != (image_embed is None) or (gauss_embed is None) != (mlp_params is None):
        raise ValueError("gauss_embed, image_embed and mlp_params go together")
    return _Rasterize.apply(means, scales, quats, opac, sh, appearance, gauss_embed, image_embed, mlp_params, lib_ctx,
                            list(cams), opts, sh_degree, segments)
