"""PyTorch autograd wrapper of the SAD render (Sec. 4.2) and its adjoint.

``sad_render_fn(params, topk_map, H, W)`` returns the rendered image
float32[H, W, 3] and is differentiable in ``params`` (float32[11, N]).  The
top-K map is a frozen, non-differentiable index set.  The forward keeps the
inputs, its output and two floats per pixel (the max logit and 1/Z of the
softmax); the backward recomputes every (pixel, site) weight from its logit
inside the CUDA adjoint instead of storing the N x K weights.  All work runs
in libsad.so through the C-ABI binding.

The adjoint writes one partial record per (site, tile) into a workspace.
When the workspace for the problem's worst case (every 16x16 tile listing
min(256 K, N) distinct sites, ``capi.sad_backward_max_records``) takes at most
``WORST_CASE_BYTES`` and half of the device's free memory, that is the one
allocated: no map can overflow it, so the backward reads no status and never
synchronises the stream.  Otherwise the workspace holds H*W*K/8 records, ten
times what a propagated top-K map of random sites needs, and a spatially
incoherent map can need more: ``CHECK_OVERFLOW`` (on by default) then reads
the workspace's record count after every backward (a stream
synchronisation); on an overflow the workspace grows to the count reported
and the backward runs again, so the gradients are always complete.  A caller
that knows its maps fit may turn the check off.
"""
from __future__ import annotations

import torch

from . import capi


CHECK_OVERFLOW = True
WORST_CASE_BYTES = 8 << 30


class _Workspaces:
    """Per-(device, problem) cache of the backward workspace: (workspace,
    whether it holds the worst case)."""

    def __init__(self):
        self._ws = {}

    def get(self, device, H, W, K, cap, min_records=0):
        key = (str(device), H, W, K, cap)
        ws, n, exact = self._ws.get(key, (None, 0, False))
        if ws is None or n < min_records:
            worst = capi.sad_backward_max_records(H, W, K, cap)
            nbytes = capi.lib().sad_backward_workspace_bytes(H, W, K, cap, worst)
            free = torch.cuda.mem_get_info(device)[0]
            if min_records == 0 and worst < 0xFFFFFFF0 and nbytes <= min(WORST_CASE_BYTES, free // 2):
                ws = capi.backward_workspace(H, W, K, cap, max_records=worst, device=device)
                n, exact = worst, True
            else:
                ws = capi.backward_workspace(H, W, K, cap, max_records=min_records, device=device)
                n, exact = min_records, False
            self._ws = {key: (ws, n, exact)}   # keep only the latest problem
        return ws, exact


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
        g = grad_rgb.contiguous().to(torch.float32)
        ws, exact = _WS.get(params.device, H, W, K, cap)
        capi.sad_render_backward_saved(params, prep, H, W, K, topk_map, g, rgb, fwd, grads, ws)
        if CHECK_OVERFLOW and not exact:
            st, used = capi.sad_workspace_status(ws)
            if st == capi.SAD_EWORKSPACE:
                # the record count is a property of the map alone: a workspace
                # of that many records holds them all on the second run
                ws, _ = _WS.get(params.device, H, W, K, cap, min_records=used)
                capi.sad_render_backward_saved(params, prep, H, W, K, topk_map, g, rgb, fwd, grads, ws)
                st, used = capi.sad_workspace_status(ws)
            if st != 0:
                raise capi.SadError(st, f"render backward: {used} partial records did not fit")
        return grads, None, None, None


def sad_render_fn(params: torch.Tensor, topk_map: torch.Tensor, H: int, W: int) -> torch.Tensor:
    """Differentiable SAD render of ``params`` over the fixed ``topk_map``."""
    return SADRender.apply(params, topk_map, H, W)
