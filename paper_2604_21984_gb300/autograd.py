"""PyTorch autograd wrapper of the SAD render (Sec. 4.2) and its adjoint.

``sad_render_fn(params, topk_map, H, W)`` returns the rendered image
float32[H, W, 3] and is differentiable in ``params`` (float32[11, N]).  The
top-K map is a frozen, non-differentiable index set.  The forward keeps the
inputs, its output and two floats per pixel (the max logit and 1/Z of the
softmax); the backward recomputes every (pixel, site) weight from its logit
inside the CUDA adjoint instead of storing the N x K weights.  All work runs
in libsad.so through the C-ABI binding.
"""
from __future__ import annotations

import torch

from . import capi


class _Workspaces:
    """Per-(device, problem) cache of the backward workspace."""

    def __init__(self):
        self._ws = {}

    def get(self, device, H, W, K, cap):
        key = (str(device), H, W, K, cap)
        ws = self._ws.get(key)
        if ws is None:
            ws = capi.backward_workspace(H, W, K, cap, device=device)
            self._ws = {key: ws}          # keep only the latest problem
        return ws


_WS = _Workspaces()


class SADRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, topk_map, H, W):
        if params.dim() != 2 or params.shape[0] != capi.N_PARAMS:
            raise ValueError("params must be float32[11, N]")
        params = params.contiguous()
        K = topk_map.shape[0] * 4
        cap = params.shape[1]
        prep = capi.empty_prep(cap, params.device)
        capi.sad_prepare_sites(params, H, W, prep)
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device=params.device)
        fwd = torch.empty((2, H * W), dtype=torch.float32, device=params.device)
        capi.sad_render_save(prep, cap, H, W, K, topk_map, rgb, fwd)
        ctx.save_for_backward(params, topk_map, prep, rgb, fwd)
        ctx.H, ctx.W, ctx.K = H, W, K
        return rgb

    @staticmethod
    def backward(ctx, grad_rgb):
        params, topk_map, prep, rgb, fwd = ctx.saved_tensors
        H, W, K = ctx.H, ctx.W, ctx.K
        cap = params.shape[1]
        grads = torch.empty_like(params)
        ws = _WS.get(params.device, H, W, K, cap)
        capi.sad_render_backward_saved(params, prep, H, W, K, topk_map,
                                       grad_rgb.contiguous().to(torch.float32), rgb, fwd, grads, ws)
        return grads, None, None, None


def sad_render_fn(params: torch.Tensor, topk_map: torch.Tensor, H: int, W: int) -> torch.Tensor:
    """Differentiable SAD render of ``params`` over the fixed ``topk_map``."""
    return SADRender.apply(params, topk_map, H, W)
