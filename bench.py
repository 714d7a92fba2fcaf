#!/usr/bin/env python3
"""Benchmark of the SAD hot path on GB300.

Headline (N=1): the differentiation workload -- torch.autograd render +
render_backward on a 2048x2048 RGB FP32 synthetic image, 262144 sites with
random SPD metrics, K=16, map from seed + 16 propagation passes.  One step =
sad_prepare_sites + sad_render_save (render keeping each pixel's max logit
and 1/Z) + sad_render_backward_saved (adjoint, exact per-site sums, chain
rule): the device work of sad_render_fn(params, map).backward(g).  Metric:
fwd+bwd Mpix/s at K=16.  The map (268 MB) is larger than L2 and is read
twice per step, so no flush is needed; steps are timed with CUDA events and
every kernel of the library by its own event pair (the library's stage
tracing) for the roofline of the dominant kernel.  `e2e` runs the same step
through sad_render_fn with the parameters and the upstream gradient uploaded
from pinned host memory and the gradients read back, every step.

Named keys and legs on one GPU (legs can be skipped):
  encode_iteration  config 2's training iteration (768x512, 32768 sites, K=16,
          J=4) as one fused sad_train_step, Mpix/s, with its own roofline;
  encode  the full config-2 encode: init + 2000 iterations with densify/prune
          every 200 (encode images/s, PSNR);
  c3      the recomputing render+backward pair, JFA warm-up and single-pass
          timings, the flood prepass, the packed render, and the recall /
          exact-match table of propagated maps vs the exact top-K;
  c4      64 uneven images (long side log-uniform 256..2048, aspect 1..1.5,
          0.06 sites/px), 500 iterations: the batched fused step in a CUDA
          graph with (K, J, tile shape) picked by the autotuner vs the plain
          one-image-at-a-time loop, equal iterations, PSNR of both;
  c5      a 120 s Poisson request stream (70% random-access decodes on
          resident site sets, 30% encodes of sides 128..4096) served with
          continuous batching vs the plain FIFO loop at 0.7x the plain loop's
          measured capacity: p50/p99, plus both on the same requests at t = 0;
  decode  random-access decode on a 1M-site resident set from the prepared
          48-byte table vs the packed 16-byte evaluation records.

With N>1 (torchrun) every rank runs its own replica of the headline workload
(weak scaling, no data-path collective); value = all pixels / max-over-ranks
time.

cpu_baseline and --impl reference: the CPU oracle (fp64 numpy render +
adjoint) on a band of rows of the headline workload over all host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing
import os
import statistics
import subprocess
import sys
import time
from concurrent.futures import ProcessPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H_C2, W_C2, N_C2, K_C2, J_C2 = 512, 768, 32768, 16, 4
H_C3, W_C3, N_C3, K_C3 = 2048, 2048, 262144, 16
METRIC = "fwd+bwd Mpix/s at K=16"
UNIT = "Mpix/s"
WORKLOAD = ("differentiation: torch.autograd render + render_backward on a 2048x2048 RGB FP32 synthetic "
            "image, 262144 sites with random SPD metrics (log-eigenvalues U[-2,2], angle U[0,pi)), "
            "radii N(0,2 px), temperatures log-uniform [0.1,10], K=16 map from seed + 16 propagation passes")
ENCODE_WORKLOAD = ("plain SAD encode training iteration: 768x512 RGB FP32 synthetic image "
                   "(value noise + 40 polygons + 1-3 px lines), 32768 gradient-weighted sites, K=16, J=4, "
                   "top-K refresh every iteration")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-encode", action="store_true", help="skip the full 2000-iteration encode leg")
    ap.add_argument("--no-c3", action="store_true", help="skip the 2048^2 render+backward leg")
    ap.add_argument("--no-c4", action="store_true", help="skip the batched-vs-plain leg")
    ap.add_argument("--no-c5", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-decode", action="store_true", help="skip the packed-decode leg")
    ap.add_argument("--no-sad1d", action="store_true", help="skip the 1-D SAD leg")
    ap.add_argument("--c3-side", type=int, default=2048,
                    help="side of the headline workload (sites at the same density); smaller sides are "
                         "for profiler captures only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--legs-only", default="", help="comma list of legs to run alone (encode,c3,c4,c5)")
    ap.add_argument("--c4-iters", type=int, default=500, help="training iterations of the c4 leg")
    ap.add_argument("--c5-seconds", type=float, default=120.0, help="length of the c5 request stream")
    ap.add_argument("--c5-max-side", type=int, default=4096, help="largest encode side in the c5 stream")
    ap.add_argument("--c5-iters", type=int, default=1000, help="iterations of each c5 encode")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# clocks sampling during the timed region
# ----------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def _gen_image(args):
    from paper_2604_21984_gb300 import inputs as gen
    H, W, seed = args
    return gen.image_noise_polygons_lines(H, W, seed=seed)


def gen_images(specs):
    """Synthetic images [(H, W, seed)] generated in parallel host processes
    (spawned, so no CUDA state is inherited)."""
    if len(specs) <= 2:
        return [_gen_image(s) for s in specs]
    workers = max(1, min(len(specs), (os.cpu_count() or 2) - 1, 16))
    with ProcessPoolExecutor(workers, mp_context=multiprocessing.get_context("spawn")) as ex:
        return list(ex.map(_gen_image, specs))


# DRAM traffic and warp instructions per launch of a timed step's dominant
# kernel, from one ncu capture of the build whose kernel sources hash to
# `sha` (profiles/).  Reported only while the sources still hash the same (a
# changed kernel has no counters until it is captured again).  The
# adjoint's capture is the 1536x1536 case of the headline workload (same
# site density), scaled to 2048x2048 by the pixel count: every term of its
# traffic is per pixel or per site (profiles/k_bwd_tile_saved_1536x1536_k16.md).
NCU_COUNTERS = {
    "k_bwd_tile": {"sources": ['sad_backward.cu', 'sad_tile.cuh', 'sad_reduce.cuh', 'sad_topk.cuh', 'sad_device.cuh'],
                   "sha": "f363d50ae2ad06d1", "dram_bytes": 459043726, "warp_inst": 354819156,
                   "captured": "1536x1536, scaled by (2048/1536)^2", "size": [2048, 2048]},
    "k_step_tile": {"sources": ['sad_step.cu', 'sad_tile.cuh', 'sad_topk.cuh', 'sad_device.cuh', 'sad_adam.cuh', 'sad_blend.cuh', 'sad_reduce.cuh'],
                    "sha": "e77352c2bd1fd65d", "dram_bytes": 34656256, "warp_inst": 114674775,
                    "captured": "768x512 (the workload itself)", "size": [512, 768]},
}
ISSUE_PEAK = 152 * 4 * 2.07e9   # warp instructions / s: 152 SMs x 4 schedulers x 1 issue/clk x 2070 MHz


def source_code_hash(files):
    """Hash of the kernels' source code without its comments and blank
    space, so that stored counters follow the code, not the comments."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2604_21984_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def ncu_counters(kernel, H, W):
    """The stored counters of `kernel` for an H x W launch: only for the
    size they were taken (or scaled) to, and only while the code is the
    captured build's."""
    c = NCU_COUNTERS.get(kernel)
    if c is None or c["size"] != [H, W]:
        return None
    return c if source_code_hash(c["sources"]) == c["sha"] else None


def reduce_max(x, dist, world, device):
    """Max over ranks of a host float (the slowest replica's time)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, units_per_rank, steps, seconds):
    """Whole-job throughput in millions of units per second: every rank
    processes its own units each step (weak scaling), the job takes as long
    as the slowest rank."""
    return world * units_per_rank * steps / seconds / 1e6


def dominant(trace):
    name = max(trace, key=lambda k: trace[k][1])
    n, ms = trace[name]
    return name, n, ms / max(n, 1)


def c3_inputs(capi, dev, seed=3000, passes=16, inject_seed=11):
    """The headline workload on the device: 262144 random anisotropic sites,
    their prepared table and a K=16 map from seed + `passes` propagation
    passes (J = 2)."""
    import torch
    from paper_2604_21984_gb300 import inputs as gen
    p = gen.sites_random_spd(H_C3, W_C3, N_C3, seed=seed)
    pt = torch.from_numpy(p).to(dev)
    prep = capi.empty_prep(N_C3, dev)
    capi.sad_prepare_sites(pt, H_C3, W_C3, prep)
    a, b = capi.empty_map(H_C3, W_C3, K_C3, dev), capi.empty_map(H_C3, W_C3, K_C3, dev)
    capi.sad_topk_seed(prep, N_C3, H_C3, W_C3, K_C3, a)
    for t in range(passes):
        s = max(1, 2048 >> (min(t, 10) + 1))
        capi.sad_update_topk(prep, N_C3, H_C3, W_C3, K_C3, a, b, (s << 16) | t, 2, inject_seed)
        a, b = b, a
    return p, pt, prep, a, b


def headline(capi, dev, args, rank, world, dist, peak, peak_kind, local):
    """The autograd pair at 2048^2, 262144 sites, K=16: one step = prepare +
    render keeping {max logit, 1/Z} + the adjoint from that state (what
    sad_render_fn(params, map).backward(g) runs on the device)."""
    import torch
    from paper_2604_21984_gb300 import inputs as gen
    from paper_2604_21984_gb300.autograd import sad_render_fn
    H, W, N, K = H_C3, W_C3, N_C3, K_C3
    P = H * W
    p, pt, prep, a, b = c3_inputs(capi, dev, seed=3000 + rank)
    del b
    g_host = torch.from_numpy(gen.grad_image(H, W, seed=3002 + rank) / P)
    g = g_host.to(dev)
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    fwd = torch.empty((2, P), dtype=torch.float32, device=dev)
    grads = torch.empty((11, N), dtype=torch.float32, device=dev)
    ws = capi.backward_workspace(H, W, K, N, device=dev)

    def step():
        capi.sad_prepare_sites(pt, H, W, prep)
        capi.sad_render_save(prep, N, H, W, K, a, rgb, fwd)
        capi.sad_render_backward_saved(pt, prep, H, W, K, a, g, rgb, fwd, grads, ws)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ws_status, records = capi.sad_workspace_status(ws)
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    evs = [(E(), E()) for _ in range(args.steps)]
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):   # the timed region: no per-kernel events between the launches
        evs[i][0].record()
        step()
        evs[i][1].record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    # the same steps once more with the library's per-kernel event pairs
    # (kernel times, launch count and the dominant kernel's roofline)
    capi.sad_trace_collect()
    capi.sad_trace_enable(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    capi.sad_trace_enable(False)
    trace = capi.sad_trace_collect()
    step_ms = [x.elapsed_time(y) for x, y in evs]
    total_ms = reduce_max(sum(step_ms), dist, world, dev)
    value = whole_job_value(world, P, args.steps, total_ms / 1e3)

    # end to end through the public API: the site parameters and the upstream
    # gradient go up from pinned host memory, sad_render_fn + backward run,
    # the parameter gradients come back, every step
    host_p = torch.from_numpy(p).pin_memory()
    host_g = g_host.pin_memory()
    host_grad = torch.empty((11, N), dtype=torch.float32).pin_memory()

    def e2e_step():
        params = host_p.to(dev, non_blocking=True).requires_grad_(True)
        gd = host_g.to(dev, non_blocking=True)
        out = sad_render_fn(params, a, H, W)
        out.backward(gd)
        host_grad.copy_(params.grad, non_blocking=True)
    for _ in range(2):
        e2e_step()
    e2e_serial_s = 0.0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e2e_serial_s += time.perf_counter() - t0
    e2e_serial_s = reduce_max(e2e_serial_s, dist, world, dev)

    # the same calls as a user's input pipeline runs them: step i + 1's
    # inputs go up on a copy stream while step i computes, and step i's
    # gradients come back on it while step i + 1 starts (every step still
    # copies its own inputs from pinned host memory and reads its gradients
    # back; the backward's workspace holds the worst case, so no step
    # synchronises the host)
    copy_s = torch.cuda.Stream(device=dev)
    comp_s = torch.cuda.current_stream(dev)
    dp = [torch.empty(host_p.shape, dtype=torch.float32, device=dev) for _ in range(2)]
    dg = [torch.empty(host_g.shape, dtype=torch.float32, device=dev) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def h2d(i):
        with torch.cuda.stream(copy_s):
            copy_s.wait_event(ev_out[i % 2])   # the buffer's previous gradient read-back is done
            dp[i % 2].copy_(host_p, non_blocking=True)
            dg[i % 2].copy_(host_g, non_blocking=True)
            ev_in[i % 2].record(copy_s)

    def piped(n):
        for e in ev_out:
            e.record(comp_s)
        h2d(0)
        for i in range(n):
            h2d(i + 1)
            comp_s.wait_event(ev_in[i % 2])
            params = dp[i % 2].requires_grad_(True)
            params.grad = None
            out = sad_render_fn(params, a, H, W)
            out.backward(dg[i % 2])
            grad = params.grad
            with torch.cuda.stream(copy_s):
                copy_s.wait_stream(comp_s)
                host_grad.copy_(grad, non_blocking=True)
                grad.record_stream(copy_s)
                ev_out[i % 2].record(copy_s)
            params.requires_grad_(False)
        torch.cuda.synchronize()
    piped(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    piped(args.steps)
    e2e_s = reduce_max(time.perf_counter() - t0, dist, world, dev)
    e2e = {"value": round(whole_job_value(world, P, args.steps, e2e_s), 3), "unit": UNIT,
           "h2d_bytes_per_step": int(host_p.numel() * 4 + host_g.numel() * 4),
           "d2h_bytes_per_step": int(host_grad.numel() * 4),
           "path": "sad_render_fn(params, map).backward(g), params and g from pinned host memory, "
                   "gradients read back; step i+1's upload and step i's read-back on a second stream",
           "serial": {"value": round(whole_job_value(world, P, args.steps, e2e_serial_s), 3),
                      "path": "the same, each step synchronised before the next upload"}}
    # roofline of the dominant kernel, from its own event pairs in the timed
    # region; algorithmic bytes per launch (per pixel and per site): render and
    # backward each read the map (4K B) and 12 B of colour or upstream
    # gradient per pixel and the 48-byte prepared record of every site
    kname, klaunch, kms = dominant(trace)
    alg = {"k_bwd_tile": P * (4 * K + 12) + 48 * N, "k_render": P * (4 * K + 12) + 48 * N}
    roofline = None
    if kname in alg:
        achieved = alg[kname] / (kms / 1e3) / 1e9
        ctr = ncu_counters(kname, H, W)
        roofline = {"kernel": kname, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                    "traffic": ctr["dram_bytes"] if ctr else None,
                    "traffic_captured": ctr["captured"] if ctr else None,
                    "algorithmic_bytes_per_launch": alg[kname],
                    "avg_launch_ms": round(kms, 5), "launches": klaunch}
        if ctr:
            ips = ctr["warp_inst"] / (kms / 1e3)
            roofline["issue"] = {"achieved_warp_inst_per_s": round(ips / 1e9, 1), "peak": round(ISSUE_PEAK / 1e9, 1),
                                 "unit": "G warp-inst/s", "frac": round(ips / ISSUE_PEAK, 4),
                                 "warp_inst_per_launch": ctr["warp_inst"]}
    pair_bytes = 2 * P * (4 * K + 12) + N * (48 + 48 + 44)
    ms = total_ms / args.steps
    pair_roof = {"bound": "hbm", "achieved": round(pair_bytes / (ms / 1e3) / 1e9, 1), "peak": peak,
                 "unit": "GB/s", "frac": round(pair_bytes / (ms / 1e3) / 1e9 / peak, 4), "peak_kind": peak_kind,
                 "algorithmic_bytes_per_step": pair_bytes}
    launches = sum(n for n, _ in trace.values())
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "sites": N, "K": K,
                   "step": "sad_prepare_sites + sad_render_save + sad_render_backward_saved",
                   "l2": "inputs larger than L2 (the 268 MB map is read twice per step), no flush",
                   "timing": "CUDA events around each step, no per-kernel events in the timed steps; "
                             "kernels_ms and the roofline from a second, traced pass of as many steps",
                   "parallelism": f"replicas x{world}"},
        "kernels_ms": {k: round(v / max(n, 1), 5) for k, (n, v) in sorted(trace.items())},
        "records_per_step": records, "ws_status": ws_status,
        "e2e": e2e, "roofline": roofline, "roofline_fwd_bwd": pair_roof, "clocks": ck,
        "gpu_launches": launches,
    }
    del rgb, fwd, grads, ws, a, prep, pt, g
    return line


def encode_iteration(capi, dev, args, rank, peak, peak_kind):
    """Config 2's training iteration as one fused sad_train_step (one-image
    batch): one propagation pass at jump 1, render + MSE + adjoint, exact
    per-site sums, Adam and the next prepared table.  Its working set fits in
    L2, so L2 is flushed (a 256 MB write) before every timed step."""
    import torch
    from paper_2604_21984_gb300 import inputs as gen
    from paper_2604_21984_gb300.encode import EncodeConfig, Encoder
    H, W, N, K, J = H_C2, W_C2, N_C2, K_C2, J_C2
    P = H * W
    img = gen.image_noise_polygons_lines(H, W, seed=2000 + rank)
    target = torch.from_numpy(img).to(dev)
    enc = Encoder(target, EncodeConfig(n_sites=N, K=K, J=J, seed=rank, densify_every=0))
    enc.init()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        enc.step()
    torch.cuda.synchronize()
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    evs = [(E(), E()) for _ in range(args.steps)]
    for i in range(args.steps):   # the timed region: no per-kernel events between the launches
        flush.zero_()
        evs[i][0].record()
        enc.step()
        evs[i][1].record()
    torch.cuda.synchronize()
    total_ms = sum(x.elapsed_time(y) for x, y in evs)
    # as many further steps with the library's per-kernel event pairs
    capi.sad_trace_collect()
    capi.sad_trace_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        enc.step()
    torch.cuda.synchronize()
    capi.sad_trace_enable(False)
    trace = capi.sad_trace_collect()
    # the same iteration as four separate calls (context for the fusion)
    enc_u = Encoder(target, EncodeConfig(n_sites=N, K=K, J=J, seed=rank, densify_every=0, fused=False))
    enc_u.init()
    for _ in range(3):
        enc_u.step()
    u_ms = []
    for _ in range(10):
        flush.zero_()
        x, y = E(), E()
        x.record()
        enc_u.step()
        y.record()
        torch.cuda.synchronize()
        u_ms.append(x.elapsed_time(y))
    del enc_u
    # end to end with host buffers: the target goes up from pinned memory and
    # the loss comes back every step
    host_img = torch.from_numpy(img).pin_memory()
    host_loss = torch.empty(1, dtype=torch.float32).pin_memory()
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        enc.target.copy_(host_img, non_blocking=True)
        enc.step()
        host_loss.copy_(enc.loss, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
    # the same iteration replayed from a CUDA graph (the batched form's
    # launch path); the traced pass's per-kernel times carry their own event
    # overhead, so they are reported beside it, not subtracted from it
    g_ms = None
    try:
        gs = torch.cuda.Stream(device=dev)
        gs.wait_stream(torch.cuda.current_stream(dev))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(gs):
            graph.capture_begin(capture_error_mode="thread_local")
            enc._call(gs)
            graph.capture_end()
            for _ in range(3):
                graph.replay()
            gev = [E() for _ in range(args.steps + 1)]
            gev[0].record(gs)
            for i in range(args.steps):
                graph.replay()
                gev[i + 1].record(gs)
        torch.cuda.synchronize()
        g_ms = statistics.median(gev[i].elapsed_time(gev[i + 1]) for i in range(args.steps))
        del graph
    except Exception as e:   # reported, the rest of the line stands
        g_ms = f"{type(e).__name__}: {e}"
    kernel_sum = sum(v / max(n, 1) for n, v in trace.values())
    kname, klaunch, kms = dominant(trace)
    alg = {"k_step_tile": P * (K * 4 * 2 + 12) + enc.cap * 48}
    roofline = None
    if kname in alg:
        achieved = alg[kname] / (kms / 1e3) / 1e9
        ctr = ncu_counters(kname, H, W)
        roofline = {"kernel": kname, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                    "traffic": ctr["dram_bytes"] if ctr else None,
                    "traffic_captured": ctr["captured"] if ctr else None,
                    "algorithmic_bytes_per_launch": alg[kname],
                    "avg_launch_ms": round(kms, 5), "launches": klaunch}
        if ctr:
            ips = ctr["warp_inst"] / (kms / 1e3)
            roofline["issue"] = {"achieved_warp_inst_per_s": round(ips / 1e9, 1), "peak": round(ISSUE_PEAK / 1e9, 1),
                                 "unit": "G warp-inst/s", "frac": round(ips / ISSUE_PEAK, 4),
                                 "warp_inst_per_launch": ctr["warp_inst"]}
    out = {"workload": ENCODE_WORKLOAD, "value": round(P * args.steps / (total_ms / 1e3) / 1e6, 3),
           "unit": UNIT, "ms_per_step": round(total_ms / args.steps, 5),
           "step": "fused sad_train_step (one-image batch)", "capacity": enc.cap,
           "l2": "flushed (256 MB write) before every timed step",
           "kernels_ms": {k: round(v / max(n, 1), 5) for k, (n, v) in sorted(trace.items())},
           "unfused_step_ms": round(statistics.median(u_ms), 5),
           "graph_replay_ms_per_step": round(g_ms, 5) if isinstance(g_ms, float) else g_ms,
           "traced_kernel_sum_ms_per_step": round(kernel_sum, 5),
           "e2e": {"value": round(P * args.steps / e2e_s / 1e6, 3), "unit": UNIT,
                   "h2d_bytes_per_step": int(host_img.numel() * 4), "d2h_bytes_per_step": 4},
           "roofline": roofline}
    del enc, flush
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    global H_C3, W_C3, N_C3, WORKLOAD
    if args.c3_side != 2048:   # a profiler case: the same workload, scaled
        H_C3 = W_C3 = args.c3_side
        N_C3 = int(round(262144 * (args.c3_side / 2048.0) ** 2))
        WORKLOAD = (WORKLOAD.replace("2048x2048", f"{H_C3}x{W_C3}").replace("262144 sites", f"{N_C3} sites")
                    + " (scaled down from 2048x2048 for a profiler capture)")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2604_21984_gb300 import build, capi
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    capi.lib()
    dev = torch.device("cuda", local)
    peak, peak_kind = measured_peaks()

    if args.legs_only:
        legs = {}
        for leg in args.legs_only.split(","):
            legs[leg] = LEGS[leg](capi, dev, peak, peak_kind, args)
        print(json.dumps(legs), flush=True)
        return

    line = headline(capi, dev, args, rank, world, dist, peak, peak_kind, local)
    torch.cuda.empty_cache()
    if world == 1:
        line["encode_iteration"] = encode_iteration(capi, dev, args, rank, peak, peak_kind)
        torch.cuda.empty_cache()
        want = [k for k in ("encode", "c3", "c4", "c5", "decode", "sad1d") if not getattr(args, "no_" + k)]
        for leg in want:
            try:
                line[leg] = LEGS[leg](capi, dev, peak, peak_kind, args)
            except Exception as e:   # a failed leg is reported, the headline still prints
                line[leg] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def encode_leg(capi, dev, peak, peak_kind, args, iters=2000):
    """The full config-2 encode: gradient-weighted init, JFA warm-up, 2000
    fused iterations with densify/prune every 200 in [200, 1800]; then the
    same encode with the candidate field refreshed every 8 iterations
    (the paper's candidate update period, App. "Candidate Field and Jump
    Schedule")."""
    import torch
    from paper_2604_21984_gb300 import inputs as gen
    from paper_2604_21984_gb300.encode import EncodeConfig, Encoder
    img = torch.from_numpy(gen.image_noise_polygons_lines(H_C2, W_C2, seed=2000)).to(dev)

    def run(**kw):
        out = None
        for rep in range(3):   # the first run warms the allocator and the library
            traced = rep == 2  # the last run sums the device time of every kernel
            if traced:
                capi.sad_trace_collect()
                capi.sad_trace_enable(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            enc = Encoder(img, EncodeConfig(n_sites=N_C2, K=K_C2, J=J_C2, iters=iters, seed=0, **kw))
            enc.run()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            if traced:
                capi.sad_trace_enable(False)
                out["gpu_kernel_seconds"] = round(sum(ms for _, ms in capi.sad_trace_collect().values()) / 1e3, 4)
            else:
                out = {"seconds": round(wall, 4), "images_per_s": round(1.0 / wall, 4),
                       "psnr_db": round(enc.psnr(), 3), "active_sites": enc.n_active}
            del enc
        return out
    res = {"workload": "768x512, 32768 gradient-weighted sites (capacity 65536), K=16, J=4, "
                       f"{iters} iterations, densify/prune every 200 in [200,1800]",
           **run(),
           "paper_context": "Kodak 768x512, 50k sites, K=8, 4000 it: 2.2 s, 46.00 dB "
                            "(Kodak @4 BPP: 40.4 dB at 2000 it, ~0.6 s); hardware not stated, "
                            "RTX 5090 implied"}
    res["cand_every_8"] = run(cand_every=8)
    res["s_grid_2"] = run(s_grid=2)   # lists on a 2x2-pixel candidate grid (separate calls)
    # refresh passes scored from the half2 candidate table, against the same
    # separate calls on the float32 table
    res["separate_calls"] = run(fused=False)
    res["cand_half2"] = run(cand_half2=True)
    # PSNR of the fused form and the two f3 variants over three seeds
    # (training is chaotic in float rounding, so one seed does not separate
    # them): seed 0 from the runs above, seeds 1 and 2 untimed
    seeds = {"fused": [res["psnr_db"]], "cand_every_8": [res["cand_every_8"]["psnr_db"]],
             "s_grid_2": [res["s_grid_2"]["psnr_db"]]}
    for sd in (1, 2):
        for name, kw in (("fused", {}), ("cand_every_8", {"cand_every": 8}), ("s_grid_2", {"s_grid": 2})):
            enc = Encoder(img, EncodeConfig(n_sites=N_C2, K=K_C2, J=J_C2, iters=iters, seed=sd, **kw))
            enc.run()
            seeds[name].append(round(enc.psnr(), 3))
            del enc
    res["psnr_over_seeds_0_1_2"] = {k: {"per_seed": v, "mean": round(statistics.mean(v), 3)}
                                    for k, v in seeds.items()}
    # the encoder's learning rates and initial temperature against their
    # neighbours (seed 0, fused): does a nearby setting do materially better?
    # And the configuration's literal rates (1e-3 positions, 5e-3 colours
    # read in normalised units) for the record.
    base_lr = EncodeConfig().lr

    def scaled(idx, f):
        return tuple(x * f if i in idx else x for i, x in enumerate(base_lr))
    sweep = {"default": res["psnr_db"], "default_lr": list(base_lr)}
    everything = range(len(base_lr))
    for name, kw in (("lr_all_x0.5", {"lr": scaled(everything, 0.5)}), ("lr_all_x2", {"lr": scaled(everything, 2.0)}),
                     ("lr_position_x0.5", {"lr": scaled((0, 1), 0.5)}), ("lr_position_x2", {"lr": scaled((0, 1), 2.0)}),
                     ("lr_radius_x0.5", {"lr": scaled((3,), 0.5)}), ("lr_radius_x2", {"lr": scaled((3,), 2.0)}),
                     ("lr_colour_x0.5", {"lr": scaled((4, 5, 6), 0.5)}), ("lr_colour_x2", {"lr": scaled((4, 5, 6), 2.0)}),
                     ("lr_log_tau_x0.5", {"lr": scaled((2,), 0.5)}), ("lr_log_tau_x2", {"lr": scaled((2,), 2.0)}),
                     ("lr_direction_aniso_x0.5", {"lr": scaled((7, 8, 9), 0.5)}),
                     ("lr_direction_aniso_x2", {"lr": scaled((7, 8, 9), 2.0)}),
                     ("tau_init_x0.5", {"tau_s_d0": 2.0}), ("tau_init_x2", {"tau_s_d0": 8.0}),
                     ("config_literal_lr", {"lr": capi.LR_CONFIG2_LITERAL})):
        enc = Encoder(img, EncodeConfig(n_sites=N_C2, K=K_C2, J=J_C2, iters=iters, seed=0, **kw))
        enc.run()
        sweep[name] = round(enc.psnr(), 3)
        del enc
    res["lr_tau_sweep_psnr_db"] = sweep
    return res


def recall_table(capi, dev, pt, prep, trials=4, n_pix=256, seed=6500):
    """Recall and exact-match of propagated maps against the exact top-K
    (sad_exact_topk, brute force over all 262144 sites) on n_pix random
    pixels per trial (the protocol of Sec. 6.5, Table "Top-K propagation
    convergence"): seed + 8 / 12 / 16 propagation passes, and the JFA flood
    prepass (seed + 11 flood passes) + 4 propagation passes.  Each trial uses
    its own injection seed and pixel sample."""
    import numpy as np
    import torch
    H, W, N, K = H_C3, W_C3, N_C3, K_C3
    rng = np.random.default_rng(seed)
    acc = {}

    def score(name, m, pix, exact):
        got = m[:, pix, :].permute(1, 0, 2).reshape(len(pix), K).cpu().numpy().view(np.uint32)
        rec, match, m8 = [], [], []
        for g_, e_ in zip(got, exact):
            es = set(int(v) for v in e_ if v != 0xFFFFFFFF)
            gs = set(int(v) for v in g_ if v != 0xFFFFFFFF)
            rec.append(len(es & gs) / max(len(es), 1))
            match.append(es == gs)
            m8.append(set(int(v) for v in g_[:8]) == set(int(v) for v in e_[:8]))
        d = acc.setdefault(name, {"recall": [], "exact_match": [], "top8_exact_match": []})
        d["recall"].append(float(np.mean(rec)))
        d["exact_match"].append(float(np.mean(match)))
        d["top8_exact_match"].append(float(np.mean(m8)))
    a, b = capi.empty_map(H, W, K, dev), capi.empty_map(H, W, K, dev)
    for tr in range(trials):
        pix_np = rng.choice(H * W, n_pix, replace=False).astype(np.int64)
        pix = torch.from_numpy(pix_np).to(dev)
        exact = capi.sad_exact_topk(prep, N, H, W, K, pix).cpu().numpy().view(np.uint32)
        capi.sad_topk_seed(prep, N, H, W, K, a)
        for t in range(16):
            s_j = max(1, 2048 >> (min(t, 10) + 1))
            capi.sad_update_topk(prep, N, H, W, K, a, b, (s_j << 16) | t, 2, 100 + tr)
            a, b = b, a
            if t + 1 in (8, 12, 16):
                score(f"passes_{t + 1}", a, pix, exact)
        capi.sad_topk_seed(prep, N, H, W, K, a)
        for t in range(11):
            capi.sad_jfa_flood(prep, N, H, W, K, a, b, ((2048 >> (t + 1)) << 16) | t)
            a, b = b, a
        for t in range(4):
            capi.sad_update_topk(prep, N, H, W, K, a, b, (1 << 16) | (100 + t), 2, 100 + tr)
            a, b = b, a
        score("flood_11_plus_4_passes", a, pix, exact)
    del a, b
    return {"protocol": f"{trials} trials x {n_pix} random pixels, exact top-{K} by brute force over "
                        f"{N} sites (sad_exact_topk), injection J=2",
            **{k: {m: round(float(np.mean(v)), 4) for m, v in d.items()} for k, d in acc.items()},
            "paper_context": "Table 'Top-K propagation convergence' (K=8, 2048^2, 16k/65k/131k sites, "
                             "another site distribution): top-8 exact match 0.981/0.987/0.987 at 8/12/16 "
                             "passes for 16k sites, 0.059/0.907/0.907 for 131k"}


def c3_leg(capi, dev, peak, peak_kind, args, iters=10):
    """The 2048^2 workload beyond the headline pair: the recomputing pair
    (sad_render + sad_render_backward, nothing kept between them), the JFA
    warm-up and single-pass timings (float32 table vs half2 candidate table),
    the flood prepass, the packed 16-byte render, and the recall table."""
    import torch
    from paper_2604_21984_gb300 import inputs as gen
    H, W, N, K = H_C3, W_C3, N_C3, K_C3
    p = gen.sites_random_spd(H, W, N, seed=3000)
    pt = torch.from_numpy(p).to(dev)
    prep = capi.empty_prep(N, dev)
    capi.sad_prepare_sites(pt, H, W, prep)
    a, b = capi.empty_map(H, W, K, dev), capi.empty_map(H, W, K, dev)
    capi.sad_topk_seed(prep, N, H, W, K, a)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in range(16):
        s = max(1, 2048 >> (min(t, 10) + 1))
        capi.sad_update_topk(prep, N, H, W, K, a, b, (s << 16) | t, 2, 11)
        a, b = b, a
    torch.cuda.synchronize()
    jfa_ms = (time.perf_counter() - t0) * 1e3
    cand = torch.empty((N, 4), dtype=torch.int32, device=dev)
    capi.sad_pack_candidates(prep, N, cand)
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn, n=10):
        for _ in range(2):
            fn()
        ev = [E() for _ in range(n + 1)]
        ev[0].record()
        for i in range(n):
            fn()
            ev[i + 1].record()
        torch.cuda.synchronize()
        return statistics.mean(ev[i].elapsed_time(ev[i + 1]) for i in range(n))
    pass_ms = {}
    for s_j in (1, 2, 4, 16, 64, 512):
        code = (s_j << 16) | 200
        pass_ms[f"f32_jump{s_j}"] = timed(lambda: capi.sad_update_topk(prep, N, H, W, K, a, b, code, 2, 11))
        pass_ms[f"half2_jump{s_j}"] = timed(lambda: capi.sad_update_topk_h2(cand, N, H, W, K, a, b, code, 2, 11))
    pass_ms["pack_candidates"] = timed(lambda: capi.sad_pack_candidates(prep, N, cand))
    del cand
    from paper_2604_21984_gb300.encode import propagate
    ha, hb = capi.empty_map(H, W, K, dev), capi.empty_map(H, W, K, dev)
    codes = [(max(1, 2048 >> (min(t, 10) + 1)) << 16) | t for t in range(16)]
    for rep in range(2):
        capi.sad_topk_seed(prep, N, H, W, K, ha)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ha, hb = propagate(prep, N, H, W, K, 2, 11, ha, hb, codes, half2_min_jump=4)
        torch.cuda.synchronize()
        jfa_h2_ms = (time.perf_counter() - t0) * 1e3
    same_h2 = float((ha == a).all(dim=2).all(dim=0).float().mean().item())   # whole lists
    del ha, hb
    fa, fb = capi.empty_map(H, W, K, dev), capi.empty_map(H, W, K, dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    capi.sad_topk_seed(prep, N, H, W, K, fa)
    for t in range(11):
        capi.sad_jfa_flood(prep, N, H, W, K, fa, fb, ((2048 >> (t + 1)) << 16) | t)
        fa, fb = fb, fa
    for t in range(4):
        capi.sad_update_topk(prep, N, H, W, K, fa, fb, (1 << 16) | (100 + t), 2, 11)
        fa, fb = fb, fa
    torch.cuda.synchronize()
    flood_ms = (time.perf_counter() - t0) * 1e3
    del fa, fb, b
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    g = torch.from_numpy(gen.grad_image(H, W, seed=3002) / (H * W)).to(dev)
    grads = torch.empty((11, N), dtype=torch.float32, device=dev)
    ws = capi.backward_workspace(H, W, K, N, device=dev)
    for _ in range(3):
        capi.sad_render(prep, N, H, W, K, a, rgb)
        capi.sad_render_backward(pt, prep, H, W, K, a, g, grads, ws)
    torch.cuda.synchronize()
    st, used = capi.sad_workspace_status(ws)
    r_ms, b_ms = [], []
    capi.sad_trace_collect()
    capi.sad_trace_enable(True)
    for _ in range(iters):
        e0, e1, e2 = E(), E(), E()
        e0.record()
        capi.sad_render(prep, N, H, W, K, a, rgb)
        e1.record()
        capi.sad_render_backward(pt, prep, H, W, K, a, g, grads, ws)
        e2.record()
        torch.cuda.synchronize()
        r_ms.append(e0.elapsed_time(e1))
        b_ms.append(e1.elapsed_time(e2))
    capi.sad_trace_enable(False)
    trace = capi.sad_trace_collect()
    words, q = capi.sad_pack_sites(pt, H, W)
    qh = q.cpu()
    rgb_p = torch.empty_like(rgb)
    for _ in range(3):
        capi.sad_render_packed(words, qh, N, H, W, K, a, rgb_p)
    pk_ms = []
    for _ in range(iters):
        e0, e1 = E(), E()
        e0.record()
        capi.sad_render_packed(words, qh, N, H, W, K, a, rgb_p)
        e1.record()
        torch.cuda.synchronize()
        pk_ms.append(e0.elapsed_time(e1))
    del a
    P = H * W
    rb = statistics.mean(r_ms)
    bb = statistics.mean(b_ms)
    render_bytes = P * (K * 4 + 12) + N * 48
    bwd_bytes = P * (K * 4 + 12) + N * (48 + 44)

    def roof(nbytes, ms):
        x = nbytes / (ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": round(x, 1), "peak": peak, "unit": "GB/s",
                "frac": round(x / peak, 4), "peak_kind": peak_kind}
    out = {
        "workload": "2048x2048, 262144 random anisotropic sites, K=16, map from seed + 16 passes",
        "recompute": {"render_ms": round(rb, 4), "backward_ms": round(bb, 4),
                      "mpix_per_s_fwd_bwd": round(P / ((rb + bb) / 1e3) / 1e6, 1),
                      "roofline_render": roof(render_bytes, rb),
                      "roofline_fwd_bwd": roof(render_bytes + bwd_bytes, rb + bb),
                      "records": used, "ws_status": st,
                      "kernels_ms": {k: round(v / max(n, 1), 5) for k, (n, v) in sorted(trace.items())}},
        "jfa_16_passes_ms": round(jfa_ms, 3),
        "flood_prepass_11_plus_4_passes_ms": round(flood_ms, 3),
        "one_pass_ms": {k: round(v, 4) for k, v in pass_ms.items()},
        "jfa_16_passes_half2_from_jump4_ms": round(jfa_h2_ms, 3),
        "jfa_half2_lists_equal_frac": round(same_h2, 4),
        "render_packed_16B_ms": round(statistics.mean(pk_ms), 4),
        "render_packed_max_abs_diff": round(float((rgb - rgb_p).abs().max().item()), 5),
    }
    del rgb, rgb_p, grads, ws, words
    torch.cuda.empty_cache()
    out["recall"] = recall_table(capi, dev, pt, prep)
    return out


def c4_leg(capi, dev, peak, peak_kind, args, n_images=64, seed=4000):
    """64 uneven images: batched fused step (CUDA graph, autotuned K/J/tile shape) vs the
    plain loop (one image at a time, the same fused kernels on a one-image
    batch, no graph), equal iterations."""
    import torch
    from paper_2604_21984_gb300 import inputs as gen
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer, autotune
    from paper_2604_21984_gb300.encode import EncodeConfig, Encoder, psnr_from_loss
    iters = args.c4_iters
    sizes = gen.batch_sizes(n_images, seed)
    t0 = time.perf_counter()
    imgs_np = gen_images([(H, W, seed + 1 + i) for i, (H, W) in enumerate(sizes)])
    gen_s = time.perf_counter() - t0
    imgs = [torch.from_numpy(a).to(dev) for a in imgs_np]
    del imgs_np
    P = sum(H * W for H, W in sizes)
    (K, J, TW), table = autotune(imgs[:8], iters=iters, seed=seed)
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    # batched
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seeds = [seed + 1 + i for i in range(n_images)]
    tr = BatchTrainer(imgs, BatchConfig(K=K, J=J, tile_w=TW), seeds=seeds)
    torch.cuda.synchronize()
    b_init = time.perf_counter() - t0
    tr.run(2)                              # graph capture outside the timed region
    torch.cuda.synchronize()
    e0, e1 = E(), E()
    e0.record()
    tr.run(iters - 2)
    e1.record()
    torch.cuda.synchronize()
    b_train = e0.elapsed_time(e1) / 1e3 * iters / (iters - 2)
    b_psnr = tr.psnr()
    del tr
    torch.cuda.empty_cache()
    # plain loop: each image alone, the fused step on a one-image batch per
    # iteration (no batching across images, no graph); at the batch's own
    # (K, J, tile) the two forms train the same trajectories (equal PSNR by
    # construction), and at K=16, J=4 for context
    def plain(pK, pJ, pTW):
        p_psnr, p_train, p_init = [], 0.0, 0.0
        for i, img in enumerate(imgs):
            H, W = sizes[i]
            n = max(1, min(H * W, int(round(0.06 * H * W))))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            enc = Encoder(img, EncodeConfig(n_sites=n, K=pK, J=pJ, capacity_factor=1.0, seed=seeds[i],
                                            densify_every=0, tile_w=pTW))
            enc.init()
            torch.cuda.synchronize()
            p_init += time.perf_counter() - t0
            e0, e1 = E(), E()
            e0.record()
            for _ in range(iters):
                enc.step()
            e1.record()
            torch.cuda.synchronize()
            p_train += e0.elapsed_time(e1) / 1e3
            p_psnr.append(psnr_from_loss(float(enc.loss.item())))
            del enc
        return {"K": pK, "J": pJ, "tile": f"{pTW}x{256 // pTW}", "train_s": round(p_train, 4),
                "init_s": round(p_init, 3), "images_per_s": round(n_images / (p_train + p_init), 3),
                "train_mpix_per_s": round(P * iters / p_train / 1e6, 1),
                "mean_psnr_db": round(statistics.mean(p_psnr), 3)}, p_train
    same, p_train = plain(K, J, TW)
    default, d_train = (same, p_train) if (K, J, TW) == (16, 4, 16) else plain(16, 4, 16)
    mb = statistics.mean(b_psnr)
    return {
        "workload": f"{n_images} images, long side log-uniform 256..2048, aspect 1..1.5, "
                    f"{P / 1e6:.1f} MP total, 0.06 sites/px, {iters} iterations",
        "autotune": {"picked": {"K": K, "J": J, "tile": f"{TW}x{256 // TW}"},
                     "sample": "the first 8 images, the same iterations",
                     "candidates": [{"K": k, "J": j, "tile": f"{tw}x{256 // tw}", "ms_per_iter": round(ms, 3),
                                     "psnr_db": round(ps, 3)} for k, j, tw, ms, ps in table]},
        "batched": {"train_s": round(b_train, 4), "init_s": round(b_init, 3),
                    "images_per_s": round(n_images / (b_train + b_init), 3),
                    "train_mpix_per_s": round(P * iters / b_train / 1e6, 1),
                    "mean_psnr_db": round(mb, 3)},
        "plain": same,
        "speedup_train": round(p_train / b_train, 3),
        "psnr_delta_db": round(mb - same["mean_psnr_db"], 3),
        "plain_k16_j4": default,
        "speedup_train_vs_k16_j4": round(d_train / b_train, 3),
        "psnr_delta_vs_k16_j4_db": round(mb - default["mean_psnr_db"], 3),
        "host_image_generation_s": round(gen_s, 2),
    }


def c5_leg(capi, dev, peak, peak_kind, args, seed=5000, details=False):
    """Poisson stream served with continuous batching vs the plain FIFO loop."""
    import numpy as np
    import torch
    from paper_2604_21984_gb300 import inputs as gen
    from paper_2604_21984_gb300.serve import (PlainLoop, Request, ServeConfig, Server, latency_summary,
                                              run_stream)
    max_side = args.c5_max_side
    res = gen.resident_sets(seed, 4)
    cfg = ServeConfig(K=16, J=4, site_pool=(sum(r[2] for r in res) + (8 << 20)),
                      pixel_pool=(sum(r[0] * r[1] for r in res) + 4 * max_side * max_side + (1 << 20)),
                      max_side=max_side, max_decode_per_tick=1 << 22)
    srv = Server(cfg, dev)
    plain = PlainLoop(cfg, dev)
    for H, W, N, sd in res:
        p = torch.from_numpy(gen.sites_random_spd(H, W, N, seed=sd)).to(dev)
        srv.add_resident(p, H, W, passes=16)
        plain.add_resident(p, H, W, passes=16)
        del p
    torch.cuda.synchronize()

    def requests(stream_specs, imgs):
        out = []
        for k, r in enumerate(stream_specs):
            if r["kind"] == "encode":
                out.append(Request("encode", arrival=r["arrival"], image=imgs[k], iters=r["iters"],
                                   seed=r["seed"] & 0x7FFFFFFF))
            else:
                H, W = res[r["resident"]][0], res[r["resident"]][1]
                xy = torch.from_numpy(gen.uniform_points(r["n"], H, W, r["seed"])).pin_memory()
                res_buf = torch.empty((r["n"], 3), dtype=torch.float32, pin_memory=True)
                out.append(Request("decode", arrival=r["arrival"], resident=r["resident"], xy=xy,
                                   out=res_buf))
        return out

    # plain capacity from a cost model: the plain loop's service time of one
    # encode (linear in pixels) and one decode (linear in coordinates), each
    # measured at two sizes, averaged over 4000 requests drawn from the
    # stream's own distribution (a short probe stream under-samples the
    # large encodes of the log-uniform side distribution)
    def service(r, img=None):
        one = requests([dict(r, arrival=0.0)], {0: img} if img is not None else {})
        run_stream(plain, one)                       # warm
        one = requests([dict(r, arrival=0.0)], {0: img} if img is not None else {})
        return run_stream(plain, one)
    enc_pts, dec_pts = [], []
    for (Hc, Wc) in ((256, 256), (768, 1024)):
        img_c = torch.from_numpy(gen_images([(Hc, Wc, 77)])[0]).to(dev)
        enc_pts.append((Hc * Wc, service(dict(kind="encode", H=Hc, W=Wc, seed=5, iters=args.c5_iters), img_c)))
    for n_c in (1000, 1000000):
        dec_pts.append((n_c, service(dict(kind="decode", resident=1, n=n_c, seed=6))))

    def fit(pts):
        (x0, y0), (x1, y1) = pts
        b = (y1 - y0) / (x1 - x0)
        return y0 - b * x0, b
    ae, be = fit(enc_pts)
    ad, bd = fit(dec_pts)
    draw = gen.serve_stream(seed + 1, 8000.0, 1.0, side=(128, max_side), iters=args.c5_iters)[:4000]
    model = [ae + be * r["H"] * r["W"] if r["kind"] == "encode" else ad + bd * r["n"] for r in draw]
    capacity = 1.0 / statistics.mean(model)
    rate = 0.7 * capacity
    spec = gen.serve_stream(seed, args.c5_seconds, rate, side=(128, max_side), iters=args.c5_iters)
    enc_idx = [k for k, r in enumerate(spec) if r["kind"] == "encode"]
    imgs = dict(zip(enc_idx, [torch.from_numpy(a).to(dev) for a in gen_images(
        [(spec[k]["H"], spec[k]["W"], spec[k]["seed"] % 100000) for k in enc_idx])]))
    out = {"workload": f"Poisson stream {args.c5_seconds} s at 0.7x plain capacity "
                       f"({rate:.2f} req/s), 70% decode (1e3..1e6 coords on 4 resident sets of "
                       f"{', '.join(str(r[2]) for r in res)} sites) / 30% encode (side 128..{max_side}, "
                       f"{args.c5_iters} iterations)",
           "plain_capacity_req_per_s": round(capacity, 3),
           "plain_service_model": {"encode_s": [round(ae, 4), f"{be:.4e} per pixel"],
                                   "decode_s": [round(ad, 5), f"{bd:.4e} per coordinate"]},
           "requests": len(spec),
           "encodes": len(enc_idx), "pool_gb": round(srv.footprint_bytes() / 1e9, 2)}
    # saturation: the same requests all at t = 0 (completion-bound throughput)
    for name, eng in (("plain", plain), ("served", srv)):
        reqs = requests([dict(r, arrival=0.0) for r in spec], imgs)
        wall = run_stream(eng, reqs)
        out.setdefault("saturated", {})[name] = {"wall_s": round(wall, 3),
                                                 "throughput_req_per_s": round(len(reqs) / wall, 3)}
        del reqs
    for name, eng in (("plain", plain), ("served", srv)):
        reqs = requests(spec, imgs)
        wall = run_stream(eng, reqs)
        s = latency_summary(reqs)
        s["wall_s"] = round(wall, 3)
        s["throughput_req_per_s"] = round(len(reqs) / wall, 3)
        ps = [10 * math.log10(3.0 / max(float(r.loss.item()), 1e-30)) for r in reqs if r.kind == "encode"]
        s["encode_mean_psnr_db"] = round(statistics.mean(ps), 3) if ps else None
        for k in ("encode", "decode"):
            if k in s:
                s[k] = {kk: (round(v, 5) if isinstance(v, float) else v) for kk, v in s[k].items()}
        if details:
            s["requests"] = [(r.kind, round(r.arrival, 4), round(r.latency, 4),
                              int(r.image.shape[0] * r.image.shape[1]) if r.kind == "encode"
                              else int(r.xy.shape[0])) for r in reqs]
        out[name] = s
        del reqs
    return out


def decode_leg(capi, dev, peak, peak_kind, args, n_query=1 << 20, n_sites=1 << 20):
    """Random-access decode on the largest config-5 resident set (1M random
    anisotropic sites, P = N/0.06): the prepared 48-byte table vs the packed
    16-byte evaluation records (App. "Data Layout and Packing")."""
    import torch
    from paper_2604_21984_gb300 import inputs as gen
    side = int(round(math.sqrt(n_sites / 0.06)))
    H = W = side
    K = 16
    pt = torch.from_numpy(gen.sites_random_spd(H, W, n_sites, seed=6000)).to(dev)
    prep = capi.empty_prep(n_sites, dev)
    capi.sad_prepare_sites(pt, H, W, prep)
    a, b = capi.empty_map(H, W, K, dev), capi.empty_map(H, W, K, dev)
    capi.sad_topk_seed(prep, n_sites, H, W, K, a)
    lb = math.ceil(math.log2(side))
    for t in range(16):
        s = max(1, (1 << lb) >> (min(t, lb - 1) + 1))
        capi.sad_update_topk(prep, n_sites, H, W, K, a, b, (s << 16) | t, 2, 11)
        a, b = b, a
    words, q = capi.sad_pack_sites(pt, H, W)
    qh = q.cpu()
    xy = torch.from_numpy(gen.uniform_points(n_query, H, W, seed=6001)).to(dev)
    r1 = torch.empty((n_query, 3), dtype=torch.float32, device=dev)
    r2 = torch.empty_like(r1)
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    res = {}
    for name, fn in (("prepared_48B", lambda: capi.sad_decode_points(prep, n_sites, H, W, K, a, xy, r1)),
                     ("packed_16B", lambda: capi.sad_decode_packed(words, qh, n_sites, H, W, K, a, xy, r2))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(10):
            e0, e1 = E(), E()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[name] = {"ms": round(statistics.median(ms), 4),
                     "mqueries_per_s": round(n_query / statistics.median(ms) / 1e3, 1)}
    return {"workload": f"{n_query} uniform queries on {n_sites} random anisotropic sites, "
                        f"{H}x{W} map from 16 passes, K=16",
            **res, "site_bytes": {"prepared": 48, "packed": 16},
            "max_abs_colour_diff_packed_vs_prepared": round(float((r1 - r2).abs().max().item()), 5)}


# SFU throughput of sm_103a: 16 exponentials per clock per SM (4 per SM
# sub-partition), the bound of the 1-D step
SFU_PEAK = 152 * 16 * 2.07e9


def sad1d_leg(capi, dev, peak, peak_kind, args, B=8192, N=64, L=1024, steps=20, fit_steps=500):
    """1-D SAD (Sec. "1D Signal Fitting"): the fused training step of a batch
    of B synthetic signals (smooth sine, step + sine, multi-frequency), L
    samples and N sites each, at K = N (every site, the paper's 64-site fits)
    and K = 16; Msamples/s of training, the PSNR after `fit_steps` steps, and
    the step's bound: every (sample, listed site) pair takes two
    exponentials (the forward and the adjoint pass), against the SFU rate."""
    import numpy as np
    import torch
    from paper_2604_21984_gb300 import inputs as gen
    y = torch.from_numpy(gen.signals_1d(B, L, seed=7000)).to(dev)
    p0 = torch.from_numpy(gen.sites_1d(y.cpu().numpy(), N)).to(dev)
    hp = capi.sad1d_hparams()
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    out = {"workload": f"{B} signals x {L} samples, {N} sites each (4 parameters), fused render + MSE + "
                       f"adjoint + Adam per step"}
    for K in (N, 16):
        p = p0.clone()
        m = torch.zeros_like(p)
        v = torch.zeros_like(p)
        loss = torch.empty(B, dtype=torch.float32, device=dev)
        t = 0
        for _ in range(3):
            t += 1
            capi.sad1d_train_step(p, m, v, B, N, L, K, y, loss, hp, t)
        torch.cuda.synchronize()
        e0, e1 = E(), E()
        e0.record()
        for _ in range(steps):
            t += 1
            capi.sad1d_train_step(p, m, v, B, N, L, K, y, loss, hp, t)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        while t < fit_steps:
            t += 1
            capi.sad1d_train_step(p, m, v, B, N, L, K, y, loss, hp, t)
        psnr = 10 * np.log10(1.0 / np.maximum(loss.cpu().numpy(), 1e-12))
        exps = 2.0 * B * L * min(K, N) / (ms / 1e3)
        out[f"K{K}"] = {"ms_per_step": round(ms, 4), "msamples_per_s": round(B * L / (ms / 1e3) / 1e6, 1),
                        "median_psnr_db_after_%d" % fit_steps: round(float(np.median(psnr)), 2),
                        "roofline": {"bound": "alu", "achieved": round(exps / 1e9, 1),
                                     "peak": round(SFU_PEAK / 1e9, 1), "unit": "G exp/s",
                                     "frac": round(exps / SFU_PEAK, 4),
                                     "peak_kind": "derived: 152 SMs x 16 SFU ops/clk x 2070 MHz"}}
    out["paper_context"] = ("64 sites x 4 params: 57.2 dB (step), 42.0 dB (multi-frequency) on the "
                            "paper's own three targets; signals here are synthetic stand-ins")
    return out


LEGS = {"encode": encode_leg, "c3": c3_leg, "c4": c4_leg, "c5": c5_leg, "decode": decode_leg,
        "sad1d": sad1d_leg}


# ----------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline key)
# ----------------------------------------------------------------------------
# The headline workload's fwd+bwd (render + adjoint, fp64 numpy oracle) on a
# band of rows of the 2048x2048 image, split over a process pool with one
# worker per host core.  Inputs come from the seeded generators only: the
# same sites, the upstream gradient, and per-pixel lists of the K
# Euclidean-nearest sites (cKDTree) standing in for the propagated map (the
# oracle's cost does not depend on which K sites are listed).

_CPU = {}


def _cpu_init(params):
    _CPU["p"] = params


def _cpu_band(args):
    from oracle import sad_oracle as oracle
    pix, ids, g = args
    H = W = H_C3
    p = _CPU["p"]
    row, col = divmod(pix, W)
    t0 = time.perf_counter()
    rgb = oracle.render(p, H, W, ids, col + 0.5, row + 0.5)
    grads = oracle.render_backward(p, H, W, ids, g, col + 0.5, row + 0.5)
    return time.perf_counter() - t0, float(rgb.sum() + grads[0].sum())


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


class CpuOracle:
    """The oracle's render + adjoint over bands of the headline workload on
    every host core (spawned workers; started before any CUDA work of the
    process is needed, and never forked after it)."""

    def __init__(self, rows_per_step):
        import numpy as np
        from paper_2604_21984_gb300 import inputs as gen
        self.np = np
        self.cores = os.cpu_count() or 1
        self.params = gen.sites_random_spd(H_C3, W_C3, N_C3, seed=3000)
        self.grad = gen.grad_image(H_C3, W_C3, seed=3002).reshape(-1, 3) / (H_C3 * W_C3)
        self.rows = rows_per_step
        self.pool = ProcessPoolExecutor(self.cores, mp_context=multiprocessing.get_context("spawn"),
                                        initializer=_cpu_init, initargs=(self.params,))
        self.bands = {}

    def _tasks(self, y0):
        np = self.np
        from paper_2604_21984_gb300 import inputs as gen
        if y0 not in self.bands:
            pix = np.arange(y0 * W_C3, (y0 + self.rows) * W_C3)
            ids = gen.knn_map(self.params, H_C3, W_C3, K_C3, seed=3001, pixels=pix)
            parts = np.array_split(np.arange(len(pix)), 4 * self.cores)
            self.bands[y0] = [(pix[q], ids[q], self.grad[pix[q]]) for q in parts if len(q)]
        return self.bands[y0]

    def step(self, y0):
        """One bounded sample: fwd+bwd of rows [y0, y0 + rows); returns wall seconds."""
        tasks = self._tasks(y0)
        t0 = time.perf_counter()
        list(self.pool.map(_cpu_band, tasks))
        return time.perf_counter() - t0

    def close(self):
        self.pool.shutdown()


def cpu_baseline(rows=512):
    """fwd+bwd Mpix/s of the oracle on a 2048 x `rows` band of the headline
    workload over all host cores (about 25 s of core time)."""
    cpu = CpuOracle(rows)
    try:
        cpu.step(0)                              # warm the workers (imports)
        el = cpu.step(768)
    finally:
        cpu.close()
    P = rows * W_C3
    return {"value": round(P / el / 1e6, 5), "unit": UNIT, "cores": cpu.cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"render + adjoint (fp64 numpy oracle) of a {W_C3}x{rows} band ({P} pixels) of the "
                      f"{W_C3}x{H_C3}, {N_C3}-site, K={K_C3} workload, lists = the K Euclidean-nearest "
                      f"sites, split over {cpu.cores} spawned worker processes, {el:.2f} s wall"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    rows = 64
    cpu = CpuOracle(rows)
    try:
        for i in range(args.warmup):
            cpu.step(rows * (i % 8))
        el = 0.0
        for i in range(args.steps):
            el += cpu.step(rows * (i % 8))
    finally:
        cpu.close()
    P = rows * W_C3
    value = P * args.steps / el / 1e6
    sample = (f"each step: render + adjoint (fp64 numpy oracle) of a {W_C3}x{rows} band ({P} pixels) of "
              f"the headline workload over {cpu.cores} host cores (spawned worker processes)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el * 1e3 / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H_C3, "W": W_C3, "sites": N_C3, "K": K_C3,
                   "parallelism": "cpu oracle"},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cpu.cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    args = parse()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
