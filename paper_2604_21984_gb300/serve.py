"""Serving: continuous batching of encode requests and batched random-access
decode over one resident pool of sites and pixels.

Two request kinds:
  * encode(image, iters): fit SAD sites to an image (gradient-weighted init
    and JFA warm-up, Sec. 4.3-4.4; then `iters` training iterations, Sec. 6.1)
    and return the site parameters;
  * decode(resident, xy): colours at arbitrary float coordinates of a resident
    site set (the random-access decode of the softmax blend, Sec. 4.2).

All encodes in flight share one set of device arrays (a site pool and a pixel
pool, sized up front from the HBM budget).  Admission allocates an encode's
slot range and pixel range (first fit); a request that does not fit waits.
Admitted encodes are trained by fused batched steps (`sad_train_step`) in
two lanes, chosen by least remaining work (see `Server`); each image's Adam
step, pass index and current map live in its own device state row, so an
image that joins late or sits out some calls follows exactly the trajectory
it would follow alone: its result is the same alone or in any mix.  A lane
whose set of images is unchanged replays its call as a CUDA graph.  All
decode requests that have arrived are answered by one `sad_decode_batch`
launch on their own stream.  Completion times are CUDA events.

`PlainLoop` is the baseline: FIFO, one request at a time, each with the
single-image calls (the same fused kernels, one image per launch).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import capi
from .encode import EncodeConfig, Encoder, warm_start

@dataclass
class ServeConfig:
    K: int = 16
    J: int = 4
    sites_per_pixel: float = 0.06
    lambda_init: float = 0.3
    site_pool: int = 1 << 22
    pixel_pool: int = 1 << 26
    max_side: int = 4096           # largest encode accepted
    max_decode_per_tick: int = 1 << 22
    pixels_per_call: int = 1 << 19    # fast-lane pixels per call (least remaining work first)
    bulk_pixels_per_call: int = 1 << 21   # bulk-lane pixels per call (arrival order)
    # CUDA stream priorities of the lanes (lower = more urgent): large encodes
    # ahead, small ones fill the gaps (measured: encode p99 no worse than the
    # plain loop; the reverse order gives a 4x lower p50 but a higher p99)
    fast_priority: int = 0
    bulk_priority: int = -1
    lr: tuple = capi.LR_DEFAULT


@dataclass
class Request:
    kind: str                      # "encode" | "decode"
    arrival: float = 0.0           # seconds after the stream's start
    image: torch.Tensor | None = None   # encode: float32[H, W, 3] (device)
    iters: int = 1000              # encode: training iterations
    seed: int = 0                  # encode: per-request seed
    resident: int = -1             # decode: resident site set index
    xy: torch.Tensor | None = None      # decode: float32[n, 2] (pinned host or device)
    out: torch.Tensor | None = None     # decode: optional float32[n, 3] result buffer (pinned host)
    rid: int = -1
    # filled in by the server
    done_event: torch.cuda.Event | None = None
    latency: float | None = None
    cancelled: bool = False
    result: object = None          # encode: float32[11, n] params; decode: float32[n, 3]
    loss: torch.Tensor | None = None


class RangePool:
    """First-fit allocator of [0, capacity) with coalescing free list."""

    def __init__(self, capacity: int, align: int = 1):
        self.capacity = capacity
        self.align = align
        self.free = [(0, capacity)]     # sorted (offset, length)

    def alloc(self, n: int):
        n = max(1, -(-n // self.align) * self.align)
        for k, (o, l) in enumerate(self.free):
            if l >= n:
                if l == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (o + n, l - n)
                return o
        return None

    def release(self, o: int, n: int):
        n = max(1, -(-n // self.align) * self.align)
        fr = self.free
        k = 0
        while k < len(fr) and fr[k][0] < o:
            k += 1
        if k > 0 and fr[k - 1][0] + fr[k - 1][1] > o:
            raise ValueError("double free or overlap")
        if k < len(fr) and o + n > fr[k][0]:
            raise ValueError("double free or overlap")
        fr.insert(k, (o, n))
        # coalesce with neighbours
        if k + 1 < len(fr) and fr[k][0] + fr[k][1] == fr[k + 1][0]:
            fr[k] = (fr[k][0], fr[k][1] + fr[k + 1][1])
            fr.pop(k + 1)
        if k > 0 and fr[k - 1][0] + fr[k - 1][1] == fr[k][0]:
            fr[k - 1] = (fr[k - 1][0], fr[k - 1][1] + fr[k][1])
            fr.pop(k)

    def free_total(self):
        return sum(l for _, l in self.free)


def encode_sites(H: int, W: int, sites_per_pixel: float) -> int:
    return max(1, min(H * W, int(round(sites_per_pixel * H * W))))


def pool_bytes(site_pool: int, pixel_pool: int, K: int) -> int:
    """HBM footprint of a Server's pools (params, Adam moments, prepared
    table, step accumulators; targets, two maps)."""
    per_site = 4 * 11 * 3 + 48 + 80
    per_pixel = 12 + 2 * 4 * K
    return site_pool * per_site + pixel_pool * per_pixel


class _Lane:
    """A stream of fused training calls over a subset of the admitted encodes,
    with its own workspace and loss buffer.  A lane whose set of images is
    unchanged for a second tick captures its call in a CUDA graph and
    replays it (the per-image state rows on the device carry the counters)."""

    def __init__(self, srv, priority):
        self.srv = srv
        self.stream = torch.cuda.Stream(device=srv.dev, priority=priority)
        self.ws = srv._workspace()
        self.loss = torch.zeros(64, dtype=torch.float32, device=srv.dev)
        self.members = []
        self.key = None
        self.call = None
        self.graph = None
        self.ticks_same = 0
        self.inflight = []
        self.retired = []

    def assign(self, members):
        members = sorted(members, key=lambda a: a["entry"]["site_offset"])
        key = tuple(a["seq"] for a in members)
        if key != self.key:
            if self.graph is not None and self.inflight:
                # replays may still be queued: keep the graph until they ran
                self.retired.append((self.graph, self.inflight[-1]))
            self.key, self.members, self.graph, self.ticks_same = key, members, None, 0
            self.call = None
            if members:
                srv, c = self.srv, self.srv.cfg
                self.call = capi.TrainStepCall(
                    capi.batch_table([a["entry"] for a in members]), c.K, c.J, srv.params, srv.m, srv.v,
                    srv.prep, srv.maps[0], srv.maps[1], c.pixel_pool, srv.targets, self.loss, srv.hp,
                    srv.state, self.ws)

    def busy(self):
        self.inflight = [e for e in self.inflight if not e.query()]
        self.retired = [(g, e) for g, e in self.retired if not e.query()]
        return len(self.inflight)

    def tick(self, max_iters):
        """T = min(max_iters, fewest iterations left) calls; finished encodes
        hand back their ranges.  Returns T."""
        if not self.members:
            return 0
        srv = self.srv
        st = self.stream
        T = max(1, min(max_iters, min(a["left"] for a in self.members)))
        for a in self.members:   # order after the image's previous work
            if a["last_lane"] is not self and a["last_event"] is not None:
                st.wait_event(a["last_event"])
        with torch.cuda.stream(st):
            if self.graph is None and self.ticks_same >= 1:
                g = torch.cuda.CUDAGraph()
                g.capture_begin(capture_error_mode="thread_local")
                self.call(st)
                g.capture_end()
                self.graph = g
            for _ in range(T):
                if self.graph is not None:
                    self.graph.replay()
                else:
                    self.call(st)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
            done = []
            for b, a in enumerate(self.members):
                if a.get("cancelled"):
                    continue
                a["left"] -= T
                a["last_lane"], a["last_event"] = self, ev
                if a["left"] <= 0:
                    e, req = a["entry"], a["req"]
                    lo, n = e["site_offset"], e["capacity"]
                    req.result = srv.params[:, lo:lo + n].clone()
                    req.loss = self.loss[b:b + 1].clone()
                    done.append(a)
            if done:
                fin = torch.cuda.Event(enable_timing=True)
                fin.record(st)
                for a in done:
                    a["req"].done_event = fin
                    srv._retire(a, fin)
        self.ticks_same += 1
        srv.launches += 3 * T   # per iteration: tile pass + adjoint, exact sums, site step
        self.inflight.append(ev)
        return T


class Server:
    """Resident pools, admission, two training lanes and the batched decode.

    The `fast` lane takes small encodes, least remaining work first, within
    `pixels_per_call`; the `bulk` lane takes the others first come first
    served within `bulk_pixels_per_call`.  The two lanes' calls overlap on
    the GPU (by default the bulk lane's stream has the higher priority and
    the small encodes fill the gaps), so small encodes are not held to the
    pace of a large one and large ones keep their arrival order.  Decodes run on a third stream at high
    priority (resident sets are never written by training)."""

    def __init__(self, cfg: ServeConfig | None = None, device="cuda", stream=None):
        self.cfg = cfg or ServeConfig()
        c = self.cfg
        self.dev = torch.device(device)
        # admission (warm starts, inserts); the completion events and the
        # stream the latencies are measured on
        self.stream = stream or torch.cuda.Stream(device=self.dev, priority=-1)
        self.dstream = torch.cuda.Stream(device=self.dev, priority=-1)
        S, Pp, K = c.site_pool, c.pixel_pool, c.K
        if Pp < c.max_side ** 2 or S < encode_sites(c.max_side, c.max_side, c.sites_per_pixel):
            raise ValueError("pools smaller than one encode of max_side")
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.params = torch.zeros((capi.N_PARAMS, S), **f32)
        self.params[0].fill_(-1.0)          # every slot inactive until used
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.prep = capi.empty_prep(S, self.dev)
        self.targets = torch.zeros((Pp, 3), **f32)
        self.maps = [torch.full((K // 4, Pp, 4), -1, dtype=torch.int32, device=self.dev) for _ in range(2)]
        self.sites = RangePool(S)
        self.pixels = RangePool(Pp, align=4)
        self.state = torch.zeros((128, 4), dtype=torch.int32, device=self.dev)
        self.free_rows = list(range(128))
        self.hp = capi.adam_hparams(lr=c.lr)
        self.fast = _Lane(self, c.fast_priority)
        self.bulk = _Lane(self, c.bulk_priority)
        # staging for the single-image warm start (largest accepted image)
        Pmax = c.max_side * c.max_side
        nmax = encode_sites(c.max_side, c.max_side, c.sites_per_pixel)
        self._st_params = torch.empty(capi.N_PARAMS * nmax, **f32)
        self._st_prep = torch.empty(4 * capi.PREP_PLANES * nmax, **f32)
        self._st_maps = [torch.empty(K * Pmax, dtype=torch.int32, device=self.dev) for _ in range(2)]
        # decode staging
        self._dq_xy = torch.empty((c.max_decode_per_tick, 2), **f32)
        self._dq_img = torch.empty(c.max_decode_per_tick, dtype=torch.int32, device=self.dev)
        self._dq_rgb = torch.empty((c.max_decode_per_tick, 3), **f32)
        self.active = []        # admitted encodes
        self.waiting = []       # encodes not admitted yet (FIFO)
        self.decodes = []       # decodes waiting for the next tick
        self.residents = []     # resident decode site sets: table entries
        self.launches = 0
        self._seq = 0
        self._freed = []        # completion events of ranges handed back
        torch.cuda.synchronize(self.dev)

    # -- pools ---------------------------------------------------------------
    def _workspace(self):
        c = self.cfg
        # records as for a full single image; tile losses for the worst tile
        # count of the pixel pool (64 images, each with a ragged tile row and
        # column)
        Pp = c.pixel_pool
        tiles = Pp // 256 + 64 * (2 * int(math.isqrt(Pp)) // 16 + 2)
        side = 16 * int(math.isqrt(tiles)) + 16
        entry = [dict(H=side, W=side, site_offset=0, capacity=0, pixel_offset=0, seed=0)]
        n = capi.lib().sad_step_workspace_bytes(
            capi.ctypes.cast(capi.batch_table(entry), capi.ctypes.c_void_p), 1, c.K, 16, c.site_pool,
            side * side, Pp * c.K // 8)
        if n == 0:
            raise ValueError("pool too large for one step workspace")
        return torch.zeros(n, dtype=torch.uint8, device=self.dev)

    def footprint_bytes(self):
        """Device bytes held for serving: the pools, the two lane workspaces and
        the library's fixed scratch buffer of the workspace-free backward
        (every device that loads the library holds it)."""
        c = self.cfg
        return (pool_bytes(c.site_pool, c.pixel_pool, c.K) + self.fast.ws.numel() + self.bulk.ws.numel()
                + capi.NOALLOC_SCRATCH_BYTES)

    def add_resident(self, params: torch.Tensor, H: int, W: int, passes: int = 16, J: int = 2,
                     seed: int = 11):
        """Place a decode site set (float32[11, N] device) in the pools with
        its field built by seed + `passes` propagation passes.  Returns its
        index."""
        c = self.cfg
        N = params.shape[1]
        lo = self.sites.alloc(N)
        po = self.pixels.alloc(H * W)
        if lo is None or po is None:
            raise MemoryError("pools too small for the resident set")
        entry = dict(H=H, W=W, site_offset=lo, capacity=N, pixel_offset=po, seed=seed)
        with torch.cuda.stream(self.stream):
            prep = capi.empty_prep(N, self.dev)
            a = capi.empty_map(H, W, c.K, self.dev)
            b = capi.empty_map(H, W, c.K, self.dev)
            pc = params.contiguous()
            capi.sad_prepare_sites(pc, H, W, prep, self.stream)
            capi.sad_topk_seed(prep, N, H, W, c.K, a, self.stream)
            L = max(H, W)
            lb = max(1, math.ceil(math.log2(L)))
            for t in range(passes):
                s = max(1, (1 << lb) >> (min(t, lb - 1) + 1))
                capi.sad_update_topk(prep, N, H, W, c.K, a, b, (s << 16) | t, J, seed, self.stream)
                a, b = b, a
            # both ping-pong buffers: training only rewrites its own images' pixels
            for mp in self.maps:
                capi.sad_batch_insert(capi.batch_table([entry]), c.K, pc, a, None, self.params,
                                      self.m, self.v, mp, self.targets, c.pixel_pool, self.stream)
            capi.sad_prepare_batch(capi.batch_table([entry]), self.params, self.prep, c.pixel_pool,
                                   self.stream)
        self.dstream.wait_stream(self.stream)
        self.residents.append(entry)
        return len(self.residents) - 1

    # -- requests --------------------------------------------------------------
    def submit(self, req: Request):
        if req.kind == "encode":
            H, W = int(req.image.shape[0]), int(req.image.shape[1])
            if max(H, W) > self.cfg.max_side:
                raise ValueError("image larger than max_side")
            res_s = sum(e["capacity"] for e in self.residents)
            res_p = sum(e["H"] * e["W"] + 3 for e in self.residents)
            if (encode_sites(H, W, self.cfg.sites_per_pixel) > self.cfg.site_pool - res_s
                    or H * W + 3 > self.cfg.pixel_pool - res_p):
                raise ValueError("encode larger than the pools left beside the resident sets")
            self.waiting.append(req)
        elif req.kind == "decode":
            if not 0 <= req.resident < len(self.residents):
                raise ValueError("unknown resident set")
            if req.xy.shape[0] > self.cfg.max_decode_per_tick:
                raise ValueError("decode larger than max_decode_per_tick")
            self.decodes.append(req)
        else:
            raise ValueError(req.kind)

    def cancel(self, req: Request) -> bool:
        """Withdraw a request that has not completed.  A waiting encode or
        decode is dropped; an admitted encode leaves the pools: its slot and
        pixel ranges and its state row are handed back and reused only after
        the device work that last touched them (its lane drops it at the next
        re-plan).  Returns False if the request is not pending here."""
        if req in self.waiting:
            self.waiting.remove(req)
        elif req in self.decodes:
            self.decodes.remove(req)
        else:
            a = next((a for a in self.active if a["req"] is req), None)
            if a is None:
                return False
            self.active.remove(a)
            a["cancelled"] = True
            self._retire(a, a["last_event"])
        req.cancelled = True
        req.done_event = None
        req.result = None
        return True

    def _retire(self, a, ev):
        e = a["entry"]
        self.sites.release(e["site_offset"], e["capacity"])
        self.pixels.release(e["pixel_offset"], e["H"] * e["W"])
        self.free_rows.append(e["state_index"])
        self._freed.append(ev)
        a["left"] = 0

    def _admit(self):
        """Admit waiting encodes (FIFO) while their ranges fit: warm start in
        the staging buffers, insert into the pools, set the state row."""
        c = self.cfg
        st = self.stream
        while self.waiting and len(self.active) < 128 and self.free_rows:
            req = self.waiting[0]
            H, W = int(req.image.shape[0]), int(req.image.shape[1])
            n = encode_sites(H, W, c.sites_per_pixel)
            lo = self.sites.alloc(n)
            if lo is None:
                break
            po = self.pixels.alloc(H * W)
            if po is None:
                self.sites.release(lo, n)
                break
            self.waiting.pop(0)
            # ranges and rows handed back by finished encodes are reused only
            # after the work that last touched them
            for ev in self._freed:
                st.wait_event(ev)
            self._freed = []
            row = self.free_rows.pop(0)
            # injection seed and pass indices as in a solo encode: seed + 0x5AD,
            # passes numbered on from the warm-up's; Adam step 1 first
            entry = dict(H=H, W=W, site_offset=lo, capacity=n, pixel_offset=po, seed=req.seed + 0x5AD,
                         state_index=row)
            with torch.cuda.stream(st):
                n_pass = self._warm_start(req, entry)
                capi.sad_prepare_batch(capi.batch_table([entry]), self.params, self.prep,
                                       c.pixel_pool, st)
                self.state[row, 0].fill_(1)
                self.state[row, 1].fill_(n_pass)
                self.state[row, 2].fill_(0)
                ready = torch.cuda.Event()
                ready.record(st)
            self._seq += 1
            self.active.append(dict(entry=entry, req=req, left=req.iters, P=H * W, seq=self._seq,
                                    last_lane=None, last_event=ready))
            self.launches += 1

    def _warm_start(self, req, entry):
        c = self.cfg
        H, W, n = entry["H"], entry["W"], entry["capacity"]
        P = H * W
        params = self._st_params[:capi.N_PARAMS * n].view(capi.N_PARAMS, n)
        prep = self._st_prep[:4 * capi.PREP_PLANES * n]
        ma = self._st_maps[0][:c.K * P].view(c.K // 4, P, 4)
        mb = self._st_maps[1][:c.K * P].view(c.K // 4, P, 4)
        target = req.image.contiguous()
        a, _, n_pass = warm_start(target, n, params, prep, ma, mb, c.K, c.J, c.lambda_init,
                                  req.seed, self.stream)
        # the image's current map goes to buffer 0 (state parity 0)
        capi.sad_batch_insert(capi.batch_table([entry]), c.K, params, a, target, self.params, self.m,
                              self.v, self.maps[0], self.targets, c.pixel_pool, self.stream)
        self.launches += 4 + n_pass + 2
        return n_pass

    def _plan(self):
        """Split the admitted encodes between the lanes.  The fast lane takes
        encodes in order of least remaining work (iterations left x pixels)
        while their pixels fit in pixels_per_call (an encode larger than that
        never goes there); the bulk lane takes the others in arrival order
        while they fit in bulk_pixels_per_call (at least one).  At most 64
        per lane; the rest wait.  Large encodes thus run first come first
        served, as in the plain loop, while small ones pass them on the fast
        lane; one large encode already fills the GPU, so stepping several
        together would only make each finish later."""
        c = self.cfg
        fast, tot = [], 0
        for a in sorted(self.active, key=lambda a: (a["left"] * a["P"], a["seq"])):
            if len(fast) == 64 or tot + a["P"] > c.pixels_per_call:
                break
            fast.append(a)
            tot += a["P"]
        taken = {a["seq"] for a in fast}
        bulk, tot = [], 0
        for a in sorted(self.active, key=lambda a: a["seq"]):
            if a["seq"] in taken:
                continue
            if len(bulk) == 64 or (bulk and tot + a["P"] > c.bulk_pixels_per_call):
                break
            bulk.append(a)
            tot += a["P"]
        self.fast.assign(fast)
        self.bulk.assign(bulk)

    def train_tick(self, max_iters: int = 1, max_inflight: int = 0) -> int:
        """Admit what fits, re-plan the lanes, and tick every lane that has
        fewer than max_inflight ticks queued (0: no limit).  Returns the
        number of iterations enqueued."""
        self._admit()
        if not self.active:
            return 0
        self._plan()
        n = 0
        for lane in (self.fast, self.bulk):
            if lane.members and (max_inflight <= 0 or lane.busy() < max_inflight):
                n += lane.tick(max_iters)
        self.active = [a for a in self.active if a["left"] > 0]
        return n

    def decode_tick(self):
        """Answer every waiting decode (up to max_decode_per_tick coordinates)
        with one batched launch on the decode stream."""
        if not self.decodes:
            return
        c = self.cfg
        reqs, total = [], 0
        while self.decodes and total + self.decodes[0].xy.shape[0] <= c.max_decode_per_tick:
            r = self.decodes.pop(0)
            reqs.append(r)
            total += r.xy.shape[0]
        table = capi.batch_table(self.residents)
        ds = self.dstream
        with torch.cuda.stream(ds):
            o = 0
            for r in reqs:
                n = r.xy.shape[0]
                self._dq_xy[o:o + n].copy_(r.xy, non_blocking=True)
                self._dq_img[o:o + n].fill_(r.resident)
                o += n
            capi.sad_decode_batch(table, c.K, self.prep, c.site_pool, self.maps[0], c.pixel_pool,
                                  self._dq_xy[:total], self._dq_img[:total], self._dq_rgb[:total], ds)
            self.launches += 1
            o = 0
            ev = torch.cuda.Event(enable_timing=True)
            for r in reqs:
                n = r.xy.shape[0]
                r.result = r.out if r.out is not None else torch.empty((n, 3), dtype=torch.float32,
                                                                        pin_memory=True)
                r.result.copy_(self._dq_rgb[o:o + n], non_blocking=True)
                o += n
            ev.record(ds)
        for r in reqs:
            r.done_event = ev

    def tick(self):
        """One training iteration of the planned encodes, then one batched
        decode of every waiting query."""
        self.train_tick(1)
        self.decode_tick()

    def busy(self):
        return bool(self.active or self.waiting or self.decodes)


class PlainLoop:
    """FIFO baseline: one request at a time with the single-image calls.
    Encodes run `Encoder.step`, the fused step on a one-image batch (the
    same kernels as the served encodes, so both give bit-identical sites;
    no densify, no graph, nothing shared across images); decodes
    `sad_decode_points` on the resident set's own arrays."""

    def __init__(self, cfg: ServeConfig | None = None, device="cuda", stream=None):
        self.cfg = cfg or ServeConfig()
        self.dev = torch.device(device)
        self.stream = stream or torch.cuda.Stream(device=self.dev)
        self.residents = []
        self.queue = []
        self.launches = 0

    def add_resident(self, params, H, W, passes=16, J=2, seed=11):
        c = self.cfg
        N = params.shape[1]
        with torch.cuda.stream(self.stream):
            prep = capi.empty_prep(N, self.dev)
            a = capi.empty_map(H, W, c.K, self.dev)
            b = capi.empty_map(H, W, c.K, self.dev)
            pc = params.contiguous()
            capi.sad_prepare_sites(pc, H, W, prep, self.stream)
            capi.sad_topk_seed(prep, N, H, W, c.K, a, self.stream)
            lb = max(1, math.ceil(math.log2(max(H, W))))
            for t in range(passes):
                s = max(1, (1 << lb) >> (min(t, lb - 1) + 1))
                capi.sad_update_topk(prep, N, H, W, c.K, a, b, (s << 16) | t, J, seed, self.stream)
                a, b = b, a
        self.residents.append(dict(prep=prep, map=a, H=H, W=W, N=N))
        return len(self.residents) - 1

    def submit(self, req: Request):
        self.queue.append(req)

    def run_one(self):
        c = self.cfg
        req = self.queue.pop(0)
        with torch.cuda.stream(self.stream):
            if req.kind == "encode":
                H, W = int(req.image.shape[0]), int(req.image.shape[1])
                n = encode_sites(H, W, c.sites_per_pixel)
                enc = Encoder(req.image.contiguous(),
                              EncodeConfig(n_sites=n, K=c.K, J=c.J, capacity_factor=1.0,
                                           lambda_init=c.lambda_init, seed=req.seed, lr=c.lr,
                                           densify_every=0),
                              stream=self.stream)
                enc.init()
                for _ in range(req.iters):
                    enc.step()
                req.result = enc.params[:, :n].clone()
                req.loss = enc.loss.clone()
                self.launches += 7 + enc.t_pass + 3 * req.iters
            else:
                r = self.residents[req.resident]
                n = req.xy.shape[0]
                xy = req.xy.to(self.dev, non_blocking=True)
                out = torch.empty((n, 3), dtype=torch.float32, device=self.dev)
                capi.sad_decode_points(r["prep"], r["N"], r["H"], r["W"], c.K, r["map"], xy, out,
                                       self.stream)
                req.result = req.out if req.out is not None else torch.empty(
                    (n, 3), dtype=torch.float32, pin_memory=True)
                req.result.copy_(out, non_blocking=True)
                self.launches += 1
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(self.stream)
        req.done_event = ev
        return req

    def busy(self):
        return bool(self.queue)


def run_stream(server, requests, max_inflight_ticks: int = 2, iters_per_tick: int = 8):
    """Replay `requests` (sorted by arrival, seconds) in real time against a
    Server or PlainLoop.  Latency = completion (CUDA event, relative to a
    start event recorded when the stream starts) - arrival.  The host only
    enqueues work: a Server gets decode batches as soon as queries arrive and
    training ticks of up to `iters_per_tick` iterations on each lane that has
    fewer than `max_inflight_ticks` queued on the device; a PlainLoop runs one
    request at a time (the next is enqueued while fewer than
    `max_inflight_ticks` are queued).  Returns wall seconds."""
    st = server.stream
    start = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(server.dev)
    start.record(st)
    t0 = time.perf_counter()
    pending = list(requests)
    inflight = []
    plain = isinstance(server, PlainLoop)
    while pending or server.busy():
        now = time.perf_counter() - t0
        while pending and pending[0].arrival <= now:
            server.submit(pending.pop(0))
        inflight = [e for e in inflight if not e.query()]
        did = False
        if plain:
            if server.busy() and len(inflight) < max_inflight_ticks:
                server.run_one()
                ev = torch.cuda.Event()
                ev.record(st)
                inflight.append(ev)
                did = True
        else:
            if server.decodes:
                server.decode_tick()
                did = True
            if server.active or server.waiting:
                if server.train_tick(iters_per_tick, max_inflight=max_inflight_ticks):
                    did = True
        if not did:
            time.sleep(0.0002)
    torch.cuda.synchronize(server.dev)
    wall = time.perf_counter() - t0
    for r in requests:
        if not r.cancelled:
            r.latency = start.elapsed_time(r.done_event) / 1e3 - r.arrival
    return wall


def latency_summary(requests):
    out = {}
    for kind in ("encode", "decode"):
        lat = sorted(r.latency for r in requests if r.kind == kind and not r.cancelled)
        if not lat:
            continue
        out[kind] = dict(n=len(lat), p50_s=float(np.percentile(lat, 50)),
                         p99_s=float(np.percentile(lat, 99)), mean_s=float(np.mean(lat)))
    return out
