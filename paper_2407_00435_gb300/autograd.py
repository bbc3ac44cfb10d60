"""torch.autograd.Function around the C-ABI forward and backward passes.

``render(scene, renderer)`` returns the (P, 3) image of all views of the
renderer's plan; its backward runs ``gs_render_backward`` and returns
gradients for means, scales, quats, opacities and SH (and, with per-level
foveation parameters, for those too).  The renderer must have been created
with ``backward=True``.
"""
from __future__ import annotations

import torch

from .gs import GS_ERR_CAPACITY, GS_OK, GsError, Renderer

_KEYS = ("means", "scales", "quats", "opac", "sh")


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opac, sh, opacity_lv, dc_lv, renderer: Renderer,
                fov: dict | None, bg, check: bool):
        sc = {"means": means.detach().contiguous(), "scales": scales.detach().contiguous(),
              "quats": quats.detach().contiguous(), "opac": opac.detach().contiguous(),
              "sh": sh.detach().contiguous()}
        f = None
        if fov is not None:
            f = dict(fov)
            f["opacity_lv"] = None if opacity_lv is None else opacity_lv.detach().contiguous()
            f["dc_lv"] = None if dc_lv is None else dc_lv.detach().contiguous()
        if check:
            renderer.fit(sc, f)
        else:
            renderer.project(sc, f)
            renderer.bin_sort()
        out = renderer.alloc_outputs(fov=f is not None)
        renderer.render(out, bg=bg, fov=f is not None)
        if check:
            code, c = renderer.counters()
            if code != GS_OK:
                raise GsError(code, "render")
        ctx.renderer = renderer
        ctx.out = out
        ctx.bg = bg
        ctx.sc = sc
        ctx.fov = f
        ctx.has_lv = (opacity_lv is not None, dc_lv is not None)
        ctx.shapes = [t.shape for t in (means, scales, quats, opac, sh)]
        return out["rgb"]

    @staticmethod
    def backward(ctx, grad_rgb):
        r: Renderer = ctx.renderer
        dev = grad_rgb.device
        grads = {k: torch.empty(ctx.sc[k].shape, device=dev) for k in _KEYS}
        if ctx.has_lv[0]:
            grads["opac_lv"] = torch.empty_like(ctx.fov["opacity_lv"])
        if ctx.has_lv[1]:
            grads["dc_lv"] = torch.empty_like(ctx.fov["dc_lv"])
        r.backward(grad_rgb.contiguous(), ctx.out, grads, bg=ctx.bg)
        return (grads["means"], grads["scales"], grads["quats"], grads["opac"], grads["sh"],
                grads.get("opac_lv"), grads.get("dc_lv"), None, None, None, None)


def render(scene: dict, renderer: Renderer, fov: dict | None = None, bg=(0.0, 0.0, 0.0),
           check: bool = True) -> torch.Tensor:
    """Differentiable render of every view of ``renderer``'s plan.

    ``scene``: dict of (N,3) means, (N,3) scales, (N,4) quats, (N,) opac,
    (N,S,3) sh device tensors (any may require grad).  ``fov``: the
    foveation dict of :func:`gs.fov_to_device` (its ``opacity_lv`` /
    ``dc_lv`` may require grad).  ``check`` synchronises once per call to
    grow the pair capacity if needed.
    """
    op_lv = fov.get("opacity_lv") if fov is not None else None
    dc_lv = fov.get("dc_lv") if fov is not None else None
    return _RenderFn.apply(scene["means"], scene["scales"], scene["quats"], scene["opac"],
                           scene["sh"], op_lv, dc_lv, renderer, fov, tuple(bg), check)


def l1_loss(rgb: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    return (rgb - target).abs().mean()


class _WeightedScaleFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scales, stats, T: float, gamma: float):
        from .gs import gs_weighted_scale
        s = scales.detach().contiguous()
        n = s.shape[0]
        ws = torch.zeros(1, dtype=torch.float64, device=s.device)
        grad = torch.zeros_like(s)
        gs_weighted_scale(n, s, stats, T, gamma, ws, grad)
        ctx.save_for_backward(grad)
        return (gamma * ws).to(scales.dtype).reshape(())

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None, None, None


def scale_decay(scales: torch.Tensor, stats: torch.Tensor, T: float, gamma: float) -> torch.Tensor:
    """gamma * WS (Sec. 3.3, Eq. 3-5): the scale-decay term of the training
    loss L = L_quality + gamma WS, from the (N, 3) activated scales and the
    (4, N) statistics of the current render (U = tiles_used, treated as a
    constant of the iterate)."""
    return _WeightedScaleFn.apply(scales, stats, float(T), float(gamma))


class _HvsqFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alt, ref, views):
        a = alt.detach().contiguous()
        r = ref.detach().contiguous()
        grad = torch.empty_like(a)
        total = torch.zeros((), dtype=torch.float64, device=a.device)
        px = 0
        for v in views:
            n = v.W * v.H
            out = torch.empty(v.n_regions, dtype=torch.float64, device=a.device)
            v(a[px:px + n], r[px:px + n], out, grad[px:px + n])
            total = total + out.sum()
            px += n
        ctx.save_for_backward(grad)
        return total.to(alt.dtype)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None, None


def hvsq_loss(alt: torch.Tensor, ref: torch.Tensor, views) -> torch.Tensor:
    """Sum over views and quality regions of HVSQ (Sec. 2.2; per region as the
    quality loss of level training, Sec. 4.3) of the (P, 3) image ``alt``
    against ``ref`` (no gradient), the views' pixels concatenated in order;
    ``views``: list of gs.HvsqView.  Differentiable in ``alt``."""
    return _HvsqFn.apply(alt, ref, list(views))
