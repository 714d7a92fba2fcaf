"""Single-image SAD encoder on the GPU (the paper's training loop, Sec. 4-6).

One encode = gradient-weighted initialisation (Sec. 4.4), a JFA warm-up of
the top-K field (seed + log2 B propagation passes, Sec. 4.3), then per
iteration: one propagation pass -> render + MSE + adjoint -> Adam (Sec. 6.1),
with a densify-then-prune event every `densify_every` iterations inside
[densify_start, densify_end] (Sec. 4.5).  With `fused` (the default) an
iteration is one `sad_train_step` call on a one-image batch (the pass and the
adjoint in one tile kernel, Adam and the next prepared table in one site
kernel); otherwise it is the four separate calls (prepare, update, train
grads, Adam), which give the same iteration.  Everything runs in libsad.so
on one CUDA stream; the host only enqueues calls (the densify event reads
back the active-site count).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from . import budget, capi


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
    lr: tuple = capi.LR_DEFAULT
    fused: bool = True   # one sad_train_step per iteration (else the separate calls)
    cand_every: int = 1  # f_cand: refresh the candidate lists every this many iterations
    cand_passes: int = 1  # n_cand: propagation passes per refresh
    prepass: str = "propagate"   # warm-up: "propagate" (jump schedule) or "flood" (JFA 3x3 prepass)
    s_grid: int = 1      # candidate grid cell size (> 1: lists per s x s cell; separate calls)
    target_bpp: float | None = None   # scale densify/prune percentiles to end near this bit rate
    tau_diffusion: float = 0.0   # lambda of the log tau gradient smoothing (> 0: separate calls)
    cand_half2: bool = False   # refresh passes score from the half2 candidate table (separate calls)
    warm_half2_jump: int = 0   # > 0: warm-up passes with at least this jump use the half2 table
    keep_grads: bool = False   # fused: also write the step's gradients to Encoder.grads
    tile_w: int = 16           # fused: adjoint tiles 16x16 (16) or 32x8 (32)
    graph: bool = False        # fused: replay the iteration and the budget events as CUDA graphs
    tau_s_d0: float = 4.0      # initial temperature: tau s d0 at the mean site spacing d0
    extra: dict = field(default_factory=dict)


def _nullctx():
    import contextlib
    return contextlib.nullcontext()


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


def warm_start(target, n0, params, prep, map_a, map_b, K, J, lambda_init, seed, stream=None,
               prepass="propagate", passes_after=4, half2_min_jump=0, tau_s_d0=4.0):
    """Gradient-weighted sites (Sec. 4.4) with tau s d0 = tau_s_d0 (4 by
    default), d0 = sqrt(P/n0),
    then the top-K field's warm-up: seed + ceil(log2 max(H, W)) propagation
    passes at the jump schedule (Sec. 4.3), or with prepass="flood" the JFA
    prepass (seed + ceil(log2 max(H, W)) 3x3 flood passes, App. "Candidate
    Field and Jump Schedule") followed by `passes_after` propagation passes
    at jump 1; injection seed `seed + 0x5AD`.  With half2_min_jump > 0 the
    propagation passes whose jump is at least that score from the half2
    candidate table (App. "Data Layout and Packing", Packed candidate
    sites): their gathers scatter, and the 16-byte record halves them.
    params: float32[11, cap] (cap >= n0; slots from n0 on inactive); prep:
    the prepared table; map_a/map_b: the two map buffers.  Returns (current
    map, other map, propagation passes run)."""
    H, W = int(target.shape[0]), int(target.shape[1])
    cap = params.shape[1]
    s = 1.0 / max(H, W)
    d0 = math.sqrt(H * W / n0)
    log_tau0 = math.log(tau_s_d0 / (s * d0))
    capi.sad_init_sites(target, n0, cap, lambda_init, seed, log_tau0, params=params, stream=stream)
    capi.sad_prepare_sites(params, H, W, prep, stream)
    capi.sad_topk_seed(prep, cap, H, W, K, map_a, stream)
    L = max(H, W)
    lb = max(1, math.ceil(math.log2(L)))
    if prepass == "flood":
        for t in range(lb):
            capi.sad_jfa_flood(prep, cap, H, W, K, map_a, map_b, jump_code(t, H, W), stream)
            map_a, map_b = map_b, map_a
        codes = [(1 << 16) | t for t in range(passes_after)]
    else:
        codes = [jump_code(t, H, W) for t in range(lb)]
    map_a, map_b = propagate(prep, cap, H, W, K, J, seed + 0x5AD, map_a, map_b, codes, stream,
                             half2_min_jump)
    return map_a, map_b, len(codes)


def propagate(prep, cap, H, W, K, J, seed, map_a, map_b, codes, stream=None, half2_min_jump=0):
    """Propagation passes with the given step codes (Sec. 4.3), ping-ponging
    map_a -> map_b; passes whose jump (code >> 16) is at least
    half2_min_jump > 0 score from the half2 candidate table.  Returns
    (current map, other map)."""
    cand = None
    if half2_min_jump > 0 and any((c >> 16) >= half2_min_jump for c in codes):
        cand = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=prep.device)
        capi.sad_pack_candidates(prep, cap, cand, stream)
    for code in codes:
        if cand is not None and (code >> 16) >= half2_min_jump:
            capi.sad_update_topk_h2(cand, cap, H, W, K, map_a, map_b, code, J, seed, stream)
        else:
            capi.sad_update_topk(prep, cap, H, W, K, map_a, map_b, code, J, seed, stream)
        map_a, map_b = map_b, map_a
    return map_a, map_b


class Encoder:
    """Fits one image.  ``target``: float32[H, W, 3] CUDA tensor in [0, 1]."""

    def __init__(self, target: torch.Tensor, cfg: EncodeConfig | None = None, stream=None):
        self.cfg = cfg or EncodeConfig()
        self.target = target.contiguous()
        self.H, self.W = int(target.shape[0]), int(target.shape[1])
        self.dev = target.device
        c = self.cfg
        if c.graph and stream is None:
            stream = torch.cuda.Stream(device=self.dev)   # graphs are captured on a side stream
        self.stream = stream
        H, W, K = self.H, self.W, c.K
        self.n0 = min(c.n_sites, H * W)
        self.cap = max(self.n0, int(math.ceil(c.capacity_factor * self.n0)))
        self.pct_scale = 1.0
        if c.target_bpp is not None:
            # the schedule simulator of Sec. 4.5: one shared scale of both
            # percentiles so that the expected final count meets the target
            tgt = budget.target_sites(c.target_bpp, H, W)
            big = max(8 * self.n0, 2 * tgt)
            self.pct_scale, _ = budget.scale_for_target(
                self.n0, tgt, c.iters, c.densify_every, c.densify_start, c.densify_end, c.densify_pct,
                c.prune_pct, big)
            trace, _ = budget.simulate_counts(self.n0, c.iters, c.densify_every, c.densify_start,
                                              c.densify_end, c.densify_pct, c.prune_pct, big,
                                              self.pct_scale)
            self.cap = max(self.cap, max([n for _, n in trace], default=self.n0) + 1)
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
        self.dp = capi.dp_params(densify_pct=min(0.95, c.densify_pct * self.pct_scale),
                                 prune_pct=min(0.95, c.prune_pct * self.pct_scale), alpha=c.alpha)
        self.t_pass = 0
        self.it = 0
        self._n_active = self.n0
        self._n_dev = torch.full((1,), self.n0, dtype=torch.int32, device=self.dev)
        self._n_dirty = False
        self._g_step = None
        self._g_dense = {}
        self.history = []
        if c.tau_diffusion > 0:
            c.fused = False   # the smoothing sits between the gradient and Adam
            self._g_tau = torch.empty(cap, dtype=torch.float32, device=self.dev)
        if c.s_grid > 1:
            # lists on the candidate grid; the per-pixel map is expanded from it
            self.Hc, self.Wc = capi.grid_dims(H, W, c.s_grid)
            self.gmaps = [torch.empty((K // 4, self.Hc * self.Wc, 4), dtype=torch.int32, device=self.dev)
                          for _ in range(2)]
            c.fused = False
        if c.cand_half2:
            if c.s_grid > 1:
                raise ValueError("cand_half2 applies to per-pixel lists (s_grid = 1)")
            self.cand = torch.empty((cap, 4), dtype=torch.int32, device=self.dev)
            c.fused = False
        if c.fused:
            self.table = capi.batch_table([dict(H=H, W=W, site_offset=0, capacity=cap, pixel_offset=0,
                                                seed=c.seed + 0x5AD)])
            self.ws_step = capi.step_workspace(self.table, K, cap, H * W, device=self.dev, tile_w=c.tile_w)
            self.state = torch.zeros((1, 4), dtype=torch.int32, device=self.dev)
            self.target_flat = self.target.reshape(-1, 3)
            self._call = None

    @property
    def map(self):
        return self.maps[0]

    def _pass(self):
        c = self.cfg
        if c.s_grid > 1:
            capi.sad_grid_update(self.prep, self.cap, self.H, self.W, c.s_grid, c.K, self.gmaps[0],
                                 self.gmaps[1], jump_code(self.t_pass, self.Hc, self.Wc), c.J,
                                 c.seed + 0x5AD, self.stream)
            self.gmaps.reverse()
            capi.sad_grid_expand(self.gmaps[0], self.H, self.W, c.s_grid, c.K, self.maps[0], self.stream)
            self.t_pass += 1
            return
        if c.cand_half2:
            capi.sad_update_topk_h2(self.cand, self.cap, self.H, self.W, c.K, self.maps[0], self.maps[1],
                                    jump_code(self.t_pass, self.H, self.W), c.J, c.seed + 0x5AD,
                                    self.stream)
        else:
            capi.sad_update_topk(self.prep, self.cap, self.H, self.W, c.K, self.maps[0], self.maps[1],
                                 jump_code(self.t_pass, self.H, self.W), c.J, c.seed + 0x5AD,
                                 self.stream)
        self.maps.reverse()
        self.t_pass += 1

    def _follow_current_stream(self):
        """Order the encoder's own stream after the work torch has queued on
        the current stream (the zero-filled arrays, the state row)."""
        if self.stream is not None:
            self.stream.wait_stream(torch.cuda.current_stream(self.dev))

    def init(self):
        """Gradient-weighted sites and the JFA warm-up of the field."""
        c = self.cfg
        self._follow_current_stream()
        if c.s_grid > 1:
            H, W = self.H, self.W
            s = 1.0 / max(H, W)
            log_tau0 = math.log(c.tau_s_d0 / (s * math.sqrt(H * W / self.n0)))
            capi.sad_init_sites(self.target, self.n0, self.cap, c.lambda_init, c.seed, log_tau0,
                                params=self.params, stream=self.stream)
            capi.sad_prepare_sites(self.params, H, W, self.prep, self.stream)
            capi.sad_grid_seed(self.prep, self.cap, H, W, c.s_grid, c.K, self.gmaps[0], self.stream)
            for _ in range(max(1, math.ceil(math.log2(max(self.Hc, self.Wc, 2))))):
                self._pass()
            return
        a, b, self.t_pass = warm_start(self.target, self.n0, self.params, self.prep, self.maps[0],
                                       self.maps[1], c.K, c.J, c.lambda_init, c.seed, self.stream,
                                       prepass=c.prepass, half2_min_jump=c.warm_half2_jump,
                                       tau_s_d0=c.tau_s_d0)
        self.maps = [a, b]
        if c.fused:
            # Adam step 1 next; pass indices continue after the warm-up's; the
            # current map is bufs[0] (state parity 0)
            with torch.cuda.stream(self.stream) if self.stream is not None else _nullctx():
                self.state.copy_(torch.tensor([[1, self.t_pass, 0, 0]], dtype=torch.int32))
            self.bufs = (self.maps[0], self.maps[1])
            self._par = 0
            self._call = capi.TrainStepCall(self.table, c.K, c.J, self.params, self.m, self.v, self.prep,
                                            self.bufs[0], self.bufs[1], self.H * self.W, self.target_flat,
                                            self.loss, self.hp, self.state, self.ws_step,
                                            grads_out=self.grads if c.keep_grads else None, tile_w=c.tile_w)
            e = dict(H=self.H, W=self.W, site_offset=0, capacity=self.cap, pixel_offset=0,
                     seed=c.seed + 0x5AD, flags=capi.STEP_KEEP_LISTS)
            self._call_keep = capi.TrainStepCall(capi.batch_table([e]), c.K, c.J, self.params, self.m,
                                                 self.v, self.prep, self.bufs[0], self.bufs[1],
                                                 self.H * self.W, self.target_flat, self.loss, self.hp,
                                                 self.state, self.ws_step,
                                                 grads_out=self.grads if c.keep_grads else None,
                                                 tile_w=c.tile_w)

    def step(self):
        """One training iteration: a candidate refresh (cand_passes passes)
        every cand_every iterations, then gradient and Adam."""
        c = self.cfg
        self.it += 1
        refresh = (self.it - 1) % max(1, c.cand_every) == 0
        if c.fused:
            if refresh:
                for _ in range(c.cand_passes - 1):
                    capi.sad_batch_update(self.table, c.K, c.J, self.prep, self.cap, self.bufs[0],
                                          self.bufs[1], self.H * self.W, self.state, self.stream)
                    self._par ^= 1
                    self.t_pass += 1
                self._call(self.stream)
                self._par ^= 1
                self.t_pass += 1
            else:
                self._call_keep(self.stream)
            self.maps = [self.bufs[self._par], self.bufs[1 - self._par]]
            return
        capi.sad_prepare_sites(self.params, self.H, self.W, self.prep, self.stream)
        if refresh:
            if c.cand_half2:   # the half2 table follows the sites (App. Packed candidate sites)
                capi.sad_pack_candidates(self.prep, self.cap, self.cand, self.stream)
            for _ in range(c.cand_passes):
                self._pass()
        capi.sad_train_grads(self.params, self.prep, self.H, self.W, c.K, self.maps[0], self.target,
                             self.grads, self.loss, self.ws, stream=self.stream)
        if c.tau_diffusion > 0:
            capi.sad_tau_diffusion(self.params, self.H, self.W, c.K, self.maps[0], c.tau_diffusion,
                                   self.grads[capi.PLANE_LOGTAU], self._g_tau, self.stream)
            self.grads[capi.PLANE_LOGTAU].copy_(self._g_tau)
        capi.sad_adam_step(self.params, self.grads, self.m, self.v, self.H, self.W, self.it, self.hp,
                           self.stream)

    @property
    def n_active(self) -> int:
        """Active sites now (reads the device count of the last budget event)."""
        if self._n_dirty:
            if self.stream is not None:
                self.stream.synchronize()
            self._n_active = int(self._n_dev.item())
            self._n_dirty = False
        return self._n_active

    def _densify_calls(self, cur_map):
        c = self.cfg
        capi.sad_prepare_sites(self.params, self.H, self.W, self.prep, self.stream)
        capi.sad_site_stats(self.prep, self.cap, self.H, self.W, c.K, cur_map, self.target,
                            self.stats, self.ws, self.stream)
        # on a candidate grid the children are found by the next passes (the
        # per-pixel map is rebuilt from the grid), so they are not seeded;
        # the event runs in stream order (no host round trip)
        capi.sad_densify_prune_async(self.params, self.m, self.v, self.H, self.W, c.K, self.stats,
                                     self.target, cur_map if c.s_grid == 1 else None, self.dp,
                                     self._n_dev, self.ws_dp, self.stream)
        if c.fused:   # the step expects the prepared table of the current sites
            capi.sad_prepare_sites(self.params, self.H, self.W, self.prep, self.stream)

    def densify(self):
        """One densify-then-prune event (Sec. 4.5), enqueued on the stream.
        With cfg.graph (fused form) the event is replayed from a CUDA graph of
        these calls, one graph per map buffer, captured at its second use."""
        c = self.cfg
        self._n_dirty = True
        if not (c.graph and c.fused):
            self._densify_calls(self.maps[0])
            return
        key = self._par
        g = self._g_dense.get(key)
        if g is None and self._g_dense.get("warm"):
            g = self._capture(lambda: self._densify_calls(self.bufs[key]))
            self._g_dense[key] = g
        if g is None:
            self._densify_calls(self.bufs[key])   # the first event also loads its kernels
            self._g_dense["warm"] = True
        else:
            with torch.cuda.stream(self.stream):   # a graph replays on the current stream
                g.replay()

    def _capture(self, calls):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(self.stream):
            g.capture_begin(capture_error_mode="thread_local")
            calls()
            g.capture_end()
        return g

    def _graph_step(self):
        """A fused iteration replayed from a CUDA graph (captured after one
        eager iteration): the per-image state row on the device carries the
        Adam step, pass index and map parity, so every replay is the next
        iteration."""
        c = self.cfg
        if c.cand_every != 1 or c.cand_passes != 1 or self.it == 0:
            return self.step()
        if self._g_step is None:
            self._g_step = self._capture(lambda: self._call(self.stream))
        self.it += 1
        with torch.cuda.stream(self.stream):   # a graph replays on the current stream
            self._g_step.replay()
        self._par ^= 1
        self.t_pass += 1
        self.maps = [self.bufs[self._par], self.bufs[1 - self._par]]

    def run(self, iters: int | None = None, log_every: int = 0):
        c = self.cfg
        n = c.iters if iters is None else iters
        if self.t_pass == 0:
            self.init()
        step = self._graph_step if (c.graph and c.fused) else self.step
        for _ in range(n):
            step()
            if (c.densify_every > 0 and c.densify_start <= self.it <= c.densify_end
                    and self.it % c.densify_every == 0):
                self.densify()
            if log_every and self.it % log_every == 0:
                self.history.append((self.it, psnr_from_loss(self._loss_value()), self.n_active))
        return self

    def render(self):
        capi.sad_prepare_sites(self.params, self.H, self.W, self.prep, self.stream)
        rgb = torch.empty((self.H, self.W, 3), dtype=torch.float32, device=self.dev)
        self._follow_current_stream()
        capi.sad_render(self.prep, self.cap, self.H, self.W, self.cfg.K, self.maps[0], rgb, self.stream)
        if self.stream is not None:
            torch.cuda.current_stream(self.dev).wait_stream(self.stream)
        return rgb

    def _loss_value(self) -> float:
        if self.stream is not None:
            self.stream.synchronize()
        return float(self.loss.item())

    def psnr(self) -> float:
        """PSNR of the current sites over the current field (the loss comes
        from the fused training kernel; gradients are discarded)."""
        capi.sad_prepare_sites(self.params, self.H, self.W, self.prep, self.stream)
        capi.sad_train_grads(self.params, self.prep, self.H, self.W, self.cfg.K, self.maps[0],
                             self.target, self.grads, self.loss, self.ws, stream=self.stream)
        return psnr_from_loss(self._loss_value())
