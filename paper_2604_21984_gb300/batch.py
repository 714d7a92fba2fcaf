"""Batched SAD training: many images of uneven sizes in one launch per stage.

All images share one set of device arrays: site parameters / Adam state /
prepared table ``[11, total_capacity]`` (image b owns a contiguous slot range),
packed targets ``[total_pixels, 3]`` and top-K map planes
``[K/4, total_pixels, 4]``.  Each image is initialised and warmed up with the
single-image calls (gradient-weighted init, JFA warm-up), copied into its
ranges (``sad_batch_insert``), and then every training iteration of the whole batch is one
``sad_train_step`` call (fused propagation + render + MSE + adjoint per tile,
exact per-site sums, Adam + prepare per site).  Each image's counters (Adam
step, pass index, current map buffer) live in a device state row advanced by
the step, so one iteration is captured once in a CUDA graph and replayed.
An image's trajectory does not depend on the rest of the batch (own site
range, seed, state row and fixed-point scale) and equals the single-image
encoder's (same seeds, same pass numbering).
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import dataclass

import torch

from . import capi
from .encode import EncodeConfig, Encoder


@dataclass
class BatchConfig:
    K: int = 16
    J: int = 4
    sites_per_pixel: float = 0.06
    lambda_init: float = 0.3
    seed: int = 0
    lr: tuple = capi.LR_DEFAULT
    graph: bool = True
    cand_every: int = 1   # f_cand: candidate refresh every this many iterations
    tile_w: int = 16      # adjoint tiles: 16 (16x16) or 32 (32x8)


class BatchTrainer:
    """Trains a list of float32[H, W, 3] CUDA images jointly."""

    def __init__(self, targets, cfg: BatchConfig | None = None, seeds=None):
        self.cfg = cfg or BatchConfig()
        c = self.cfg
        if not 1 <= len(targets) <= 64:
            raise ValueError("1..64 images per batch")
        self.dev = targets[0].device
        self.images = []
        site, pix = 0, 0
        for b, t in enumerate(targets):
            H, W = int(t.shape[0]), int(t.shape[1])
            n = max(1, min(H * W, int(round(c.sites_per_pixel * H * W))))
            sd = seeds[b] if seeds is not None else c.seed * 1000003 + b + 1
            # table seed = injection seed of the training passes (the
            # single-image encoder's convention: user seed + 0x5AD)
            self.images.append(dict(H=H, W=W, site_offset=site, capacity=n, pixel_offset=pix,
                                    seed=sd + 0x5AD, user_seed=sd, n=n))
            site += n
            pix += H * W
        self.total_cap, self.total_pixels = site, pix
        self.table = capi.batch_table(self.images)
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.params = torch.empty((capi.N_PARAMS, site), **f32)
        self.m = torch.empty_like(self.params)
        self.v = torch.empty_like(self.params)
        self.prep = capi.empty_prep(site, self.dev)
        self.targets = torch.empty((pix, 3), **f32)
        K = c.K
        self.bufs = [torch.empty((K // 4, pix, 4), dtype=torch.int32, device=self.dev) for _ in range(2)]
        self.loss = torch.zeros(len(targets), **f32)
        self.state = torch.zeros((len(targets), 4), dtype=torch.int32, device=self.dev)
        self.hp = capi.adam_hparams(lr=c.lr)
        self.ws = capi.step_workspace(self.table, K, site, pix, device=self.dev, tile_w=c.tile_w)
        self.graph = None
        self.steps = 0
        self.refreshes = 0
        self._init(targets)
        self._call = capi.TrainStepCall(self.table, c.K, c.J, self.params, self.m, self.v, self.prep,
                                        self.bufs[0], self.bufs[1], self.total_pixels, self.targets,
                                        self.loss, self.hp, self.state, self.ws, tile_w=c.tile_w)
        keep = capi.batch_table([dict(im, flags=capi.STEP_KEEP_LISTS) for im in self.images])
        self._call_keep = capi.TrainStepCall(keep, c.K, c.J, self.params, self.m, self.v, self.prep,
                                             self.bufs[0], self.bufs[1], self.total_pixels, self.targets,
                                             self.loss, self.hp, self.state, self.ws, tile_w=c.tile_w)

    @property
    def maps(self):
        """[current map buffer, other] (every image refreshes on the same
        calls, so all share the parity of the refresh count)."""
        p = self.refreshes & 1
        return [self.bufs[p], self.bufs[1 - p]]

    def _init(self, targets):
        c = self.cfg
        for b, (t, im) in enumerate(zip(targets, self.images)):
            H, W, lo, n, po = im["H"], im["W"], im["site_offset"], im["capacity"], im["pixel_offset"]
            enc = Encoder(t.contiguous(), EncodeConfig(n_sites=n, K=c.K, J=c.J, capacity_factor=1.0,
                                                       lambda_init=c.lambda_init,
                                                       seed=im["user_seed"]))
            enc.init()
            # training pass indices continue after the image's warm-up passes,
            # as in the single-image encoder
            im["state_index"] = b
            im["n_pass"] = enc.t_pass
            capi.sad_batch_insert(capi.batch_table([im]), c.K, enc.params, enc.maps[0], t.contiguous(),
                                  self.params, self.m, self.v, self.bufs[0], self.targets,
                                  self.total_pixels)
            del enc
        self.table = capi.batch_table(self.images)
        capi.sad_prepare_batch(self.table, self.params, self.prep, self.total_pixels)
        # state rows: Adam step 1, passes numbered on from the warm-up's, map in bufs[0]
        self.state.copy_(torch.tensor([[1, im["n_pass"], 0, 0] for im in self.images], dtype=torch.int32))

    def _step(self, stream=None):
        """One iteration: a candidate refresh on the first of every
        cand_every iterations, the current lists on the others."""
        if self.steps % max(1, self.cfg.cand_every) == 0:
            self._call(stream)
            self.refreshes += 1
        else:
            self._call_keep(stream)
        self.steps += 1

    def _capture(self):
        """One candidate period (cand_every iterations) in a CUDA graph: the
        calls never change, the state rows on the device carry the counters
        and the map parity."""
        s = torch.cuda.Stream(device=self.dev)
        s.wait_stream(torch.cuda.current_stream(self.dev))
        g = torch.cuda.CUDAGraph()
        steps, refreshes = self.steps, self.refreshes
        with torch.cuda.stream(s):
            # capture records the calls without running them
            with torch.cuda.graph(g, stream=s):
                for _ in range(max(1, self.cfg.cand_every)):
                    self._step(s)
        self.steps, self.refreshes = steps, refreshes
        torch.cuda.current_stream(self.dev).wait_stream(s)
        self.graph = g

    def run(self, iters: int):
        """`iters` training iterations of every image (graph replays of whole
        candidate periods when on, single calls for the rest)."""
        F = max(1, self.cfg.cand_every)
        if self.cfg.graph:
            while iters > 0 and self.steps % F != 0:
                self._step()
                iters -= 1
            if iters >= F:
                if self.graph is None:
                    self._capture()
                for _ in range(iters // F):
                    self.graph.replay()
                self.steps += F * (iters // F)
                self.refreshes += iters // F
                iters -= F * (iters // F)
        for _ in range(iters):
            self._step()
        return self

    def map_for(self, b):
        """Current map of image b with image-local site ids (uint32 numpy [P, K])."""
        im = self.images[b]
        po, P, lo = im["pixel_offset"], im["H"] * im["W"], im["site_offset"]
        ids = capi.ids_from_map(self.maps[0][:, po:po + P].contiguous()).astype("int64")
        import numpy as np
        return np.where(ids == 0xFFFFFFFF, ids, ids - lo).astype(np.uint32)

    def psnr(self):
        """Per-image PSNR from the losses of the last step."""
        return [float("inf") if l <= 0 else 10 * math.log10(3.0 / l) for l in self.loss.tolist()]


def tune_key(image_sizes, iters, candidates, psnr_tol, sites_per_pixel, device_name):
    """Cache key of an autotuner decision: the batch's image sizes (sorted),
    the iteration budget, the candidates, the PSNR tolerance, the site
    density and the GPU."""
    return json.dumps({"images": sorted([int(h), int(w)] for h, w in image_sizes), "iters": int(iters),
                       "candidates": [list(map(int, c)) for c in candidates], "psnr_tol": float(psnr_tol),
                       "sites_per_pixel": float(sites_per_pixel), "gpu": str(device_name)}, sort_keys=True)


def cache_load(path, key):
    """The cached decision for key, or None (a missing or unreadable file is
    an empty cache)."""
    try:
        with open(path) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def cache_store(path, key, value):
    """Add key -> value to the JSON cache file (written whole, then renamed)."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[key] = value
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


TUNE_CANDIDATES = ((16, 4, 16), (16, 4, 32), (16, 2, 16), (8, 4, 16), (8, 4, 32), (8, 2, 16))


def autotune(targets, iters: int = 100, candidates=TUNE_CANDIDATES, psnr_tol: float = 0.05,
             seed: int = 0, cache_path: str | None = None):
    """Pick (K, J, tile width) for a batch: each candidate (a (K, J) pair
    means tile width 16) trains `targets` (a sample of the batch) for
    `iters` iterations, the intended budget, so that the PSNR compared is
    the one the job will reach; the pick is the fastest candidate whose
    (K, J) reaches a mean PSNR (over its tile shapes) within psnr_tol dB of
    the best (K, J).  With cache_path, the decision
    is read from / written to a JSON cache keyed by tune_key.  Returns (best
    (K, J, tile_w), table of (K, J, tile_w, ms per iteration, mean PSNR))."""
    candidates = tuple(tuple(c) if len(c) == 3 else (c[0], c[1], 16) for c in candidates)
    key = None
    if cache_path is not None:
        key = tune_key([t.shape[:2] for t in targets], iters, candidates, psnr_tol,
                       BatchConfig().sites_per_pixel, torch.cuda.get_device_name(targets[0].device))
        hit = cache_load(cache_path, key)
        if hit is not None:
            return tuple(hit["pick"]), [tuple(r) for r in hit["table"]]
    rows = []
    for K, J, TW in candidates:
        tr = BatchTrainer(targets, BatchConfig(K=K, J=J, seed=seed, tile_w=TW))
        n_t = min(10, max(1, iters // 4))
        tr.run(iters - n_t)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tr.run(n_t)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / n_t
        p = sum(tr.psnr()) / len(targets)
        rows.append((K, J, TW, ms, p))
        del tr
    # the tile shape changes the computation only by rounding, so the
    # quality of a candidate is that of its (K, J): the mean PSNR over its
    # tile shapes (one trajectory's PSNR moves by a few hundredths of a dB
    # under any change of rounding)
    groups = {}
    for r in rows:
        groups.setdefault((r[0], r[1]), []).append(r[4])
    quality = {kj: sum(v) / len(v) for kj, v in groups.items()}
    best_q = max(quality.values())
    ok = [r for r in rows if quality[(r[0], r[1])] >= best_q - psnr_tol]
    best = min(ok, key=lambda r: r[3])
    if key is not None:
        cache_store(cache_path, key, {"pick": list(best[:3]), "table": [list(r) for r in rows]})
    return tuple(best[:3]), rows
