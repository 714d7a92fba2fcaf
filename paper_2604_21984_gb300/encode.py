"""Single-image SAD encoder on the GPU (the paper's training loop, Sec. 4-6).

One encode = gradient-weighted initialisation (Sec. 4.4), a JFA warm-up of
the top-K field (seed + log2 B propagation passes, Sec. 4.3), then per
iteration: prepare sites -> one propagation pass -> fused render + MSE +
adjoint -> Adam (Sec. 6.1), with a densify-then-prune event every
`densify_every` iterations inside [densify_start, densify_end] (Sec. 4.5).
Everything runs in libsad.so on one CUDA stream; the host only enqueues
calls (the densify event reads back the active-site count).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from . import capi


@dataclass
class EncodeConfig:
    n_sites: int = 32768
    K: int = 16
    J: int = 4
    iters: int = 2000
    lambda_init: float = 0.3
    capacity_factor: float = 2.0
    densify_every: int = 200
    densify_start: int = 200
    densify_end: int = 1800
    densify_pct: float = 0.01
    prune_pct: float = 0.033
    alpha: float = 0.7
    seed: int = 0
    lr: tuple = (1e-3, 1e-3, 1e-2, 1e-3, 5e-3, 5e-3, 5e-3, 1e-2, 1e-2, 1e-2, 0.0)
    extra: dict = field(default_factory=dict)


def jump_code(t: int, H: int, W: int) -> int:
    """Step parameter of pass t: jump s_t = max(1, B / 2^(min(t, log2 B - 1) + 1))
    in the high 16 bits, t in the low 16 bits (Sec. 4.3; App. step encoding)."""
    L = max(H, W)
    lb = math.ceil(math.log2(L)) if L > 1 else 0
    s = max(1, (1 << lb) >> (min(t, lb - 1) + 1)) if lb > 0 else 1
    return ((s & 0xFFFF) << 16) | (t & 0xFFFF)


def psnr_from_loss(loss: float) -> float:
    """PSNR of images in [0,1] from L = mean over pixels of |c - I|^2 (3 channels)."""
    mse = loss / 3.0
    return float("inf") if mse <= 0 else 10.0 * math.log10(1.0 / mse)


class Encoder:
    """Fits one image.  ``target``: float32[H, W, 3] CUDA tensor in [0, 1]."""

    def __init__(self, target: torch.Tensor, cfg: EncodeConfig | None = None, stream=None):
        self.cfg = cfg or EncodeConfig()
        self.target = target.contiguous()
        self.H, self.W = int(target.shape[0]), int(target.shape[1])
        self.dev = target.device
        self.stream = stream
        c = self.cfg
        H, W, K = self.H, self.W, c.K
        self.n0 = min(c.n_sites, H * W)
        self.cap = max(self.n0, int(math.ceil(c.capacity_factor * self.n0)))
        cap = self.cap
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.params = torch.empty((capi.N_PARAMS, cap), **f32)
        self.m = torch.zeros((capi.N_PARAMS, cap), **f32)
        self.v = torch.zeros((capi.N_PARAMS, cap), **f32)
        self.grads = torch.empty((capi.N_PARAMS, cap), **f32)
        self.stats = torch.empty((8, cap), **f32)
        self.loss = torch.zeros(1, **f32)
        self.prep = capi.empty_prep(cap, self.dev)
        self.maps = [capi.empty_map(H, W, K, self.dev), capi.empty_map(H, W, K, self.dev)]
        self.ws = capi.backward_workspace(H, W, K, cap, device=self.dev)
        self.ws_dp = capi.densify_workspace(cap, H, W, self.dev)
        self.hp = capi.adam_hparams(lr=c.lr)
        self.dp = capi.dp_params(densify_pct=c.densify_pct, prune_pct=c.prune_pct, alpha=c.alpha)
        self.t_pass = 0
        self.it = 0
        self.n_active = self.n0
        self.history = []

    @property
    def map(self):
        return self.maps[0]

    def _pass(self):
        c = self.cfg
        capi.sad_update_topk(self.prep, self.cap, self.H, self.W, c.K, self.maps[0], self.maps[1],
                             jump_code(self.t_pass, self.H, self.W), c.J, c.seed + 0x5AD,
                             self.stream)
        self.maps.reverse()
        self.t_pass += 1

    def init(self):
        """Gradient-weighted sites, tau s d0 = 4 with d0 = sqrt(P/N), and the
        JFA warm-up of the field."""
        c = self.cfg
        H, W = self.H, self.W
        s = 1.0 / max(H, W)
        d0 = math.sqrt(H * W / self.n0)
        log_tau0 = math.log(4.0 / (s * d0))
        capi.sad_init_sites(self.target, self.n0, self.cap, c.lambda_init, c.seed, log_tau0,
                            params=self.params, stream=self.stream)
        capi.sad_prepare_sites(self.params, H, W, self.prep, self.stream)
        capi.sad_topk_seed(self.prep, self.cap, H, W, c.K, self.maps[0], self.stream)
        L = max(H, W)
        for _ in range(max(1, math.ceil(math.log2(L)))):
            self._pass()

    def step(self):
        """One training iteration (prepare, 1 pass, fused gradient, Adam)."""
        c = self.cfg
        self.it += 1
        capi.sad_prepare_sites(self.params, self.H, self.W, self.prep, self.stream)
        self._pass()
        capi.sad_train_grads(self.params, self.prep, self.H, self.W, c.K, self.maps[0], self.target,
                             self.grads, self.loss, self.ws, stream=self.stream)
        capi.sad_adam_step(self.params, self.grads, self.m, self.v, self.H, self.W, self.it, self.hp,
                           self.stream)

    def densify(self):
        c = self.cfg
        capi.sad_prepare_sites(self.params, self.H, self.W, self.prep, self.stream)
        capi.sad_site_stats(self.prep, self.cap, self.H, self.W, c.K, self.maps[0], self.target,
                            self.stats, self.ws, self.stream)
        self.n_active = capi.sad_densify_prune(self.params, self.m, self.v, self.H, self.W, c.K,
                                               self.stats, self.target, self.maps[0], self.dp,
                                               self.ws_dp, self.stream)
        return self.n_active

    def run(self, iters: int | None = None, log_every: int = 0):
        c = self.cfg
        n = c.iters if iters is None else iters
        if self.t_pass == 0:
            self.init()
        for _ in range(n):
            self.step()
            if (c.densify_every > 0 and c.densify_start <= self.it <= c.densify_end
                    and self.it % c.densify_every == 0):
                self.densify()
            if log_every and self.it % log_every == 0:
                self.history.append((self.it, psnr_from_loss(float(self.loss.item())), self.n_active))
        return self

    def render(self):
        capi.sad_prepare_sites(self.params, self.H, self.W, self.prep, self.stream)
        rgb = torch.empty((self.H, self.W, 3), dtype=torch.float32, device=self.dev)
        capi.sad_render(self.prep, self.cap, self.H, self.W, self.cfg.K, self.maps[0], rgb, self.stream)
        return rgb

    def psnr(self) -> float:
        """PSNR of the current sites over the current field (the loss comes
        from the fused training kernel; gradients are discarded)."""
        capi.sad_prepare_sites(self.params, self.H, self.W, self.prep, self.stream)
        capi.sad_train_grads(self.params, self.prep, self.H, self.W, self.cfg.K, self.maps[0],
                             self.target, self.grads, self.loss, self.ws, stream=self.stream)
        return psnr_from_loss(float(self.loss.item()))
