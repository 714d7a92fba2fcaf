#!/usr/bin/env python3
"""Benchmark of the SAD hot path (one training iteration) on GB300.

Workload (N=1): plain SAD encode step of one 768x512 RGB FP32 synthetic image
(multi-octave value noise + 40 polygons + thin lines), 32768 sites, K=16,
J=4 injected ids, after a JFA warm-up of the top-K field.  One step = one
training iteration of the hot path, all on the GPU:
    sad_prepare_sites -> sad_update_topk (1 pass, jump 1)
    -> sad_train_grads (fused render + MSE + adjoint + segmented reduce)
    -> sad_adam_step.
Metric: fwd+bwd Mpix/s at K=16 (pixels of training iterations per second).
The step's working set (~60 MB) fits in L2, so L2 is flushed (a 256 MB write)
before every timed step and each step is timed alone with CUDA events.

With N>1 (torchrun) every rank trains its own image (weak scaling, no
data-path collective); value = all pixels / max-over-ranks time.

Also measured: render + backward at 2048x2048, 262144 sites, K=16 (the
autograd form) for the HBM roofline of the backward.

--impl reference runs the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H_C2, W_C2, N_C2, K_C2, J_C2 = 512, 768, 32768, 16, 4
METRIC = "fwd+bwd Mpix/s at K=16"
UNIT = "Mpix/s"
WORKLOAD = ("plain SAD encode training iteration: 768x512 RGB FP32 synthetic image "
            "(value noise + 40 polygons + 1-3 px lines), 32768 sites, K=16, J=4, "
            "top-K refresh every iteration")
LAUNCHES_PER_STEP = 11   # prepare, topk update, bwd tile, loss, seg count, 3 scan, scatter, site grads, adam


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-c3", action="store_true", help="skip the 2048^2 render+backward leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--only-c3", action="store_true",
                    help="run only the 2048^2 render+backward leg (profiling target)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# workload inputs (seeded, host side)
# ----------------------------------------------------------------------------

def c2_inputs(rank):
    from paper_2604_21984_gb300 import inputs as gen
    img = gen.image_noise_polygons_lines(H_C2, W_C2, seed=2000 + rank)
    s = 1.0 / max(H_C2, W_C2)
    d0 = math.sqrt(H_C2 * W_C2 / N_C2)
    tau0 = 4.0 / (s * d0)                      # tau s d0 = 4: a few px of soft overlap
    params = gen.sites_isotropic(img, N_C2, seed=2100 + rank, scale_px=1.0, tau=tau0)
    return img, params


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

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

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

    if args.only_c3:
        peak, peak_kind = measured_peaks()
        print(json.dumps({"c3_render_backward": c3_leg(capi, torch.device("cuda", local), peak, peak_kind)}))
        return
    H, W, N, K, J = H_C2, W_C2, N_C2, K_C2, J_C2
    P = H * W
    img, params = c2_inputs(rank)
    dev = torch.device("cuda", local)
    pt = torch.from_numpy(params).to(dev)
    target = torch.from_numpy(img).to(dev)
    prep = capi.empty_prep(N, dev)
    ma, mb = capi.empty_map(H, W, K, dev), capi.empty_map(H, W, K, dev)
    grads = torch.empty((11, N), dtype=torch.float32, device=dev)
    m = torch.zeros_like(pt)
    v = torch.zeros_like(pt)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    ws = capi.backward_workspace(H, W, K, N, device=dev)
    hp = capi.adam_hparams()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step_code(t):
        L = max(H, W)
        lb = math.ceil(math.log2(L))
        s = max(1, (1 << lb) >> (min(t, lb - 1) + 1))
        return (s << 16) | (t & 0xFFFF)

    # JFA warm-up of the field: seed + log2(B) passes
    capi.sad_prepare_sites(pt, H, W, prep)
    capi.sad_topk_seed(prep, N, H, W, K, ma)
    t_pass = 0
    for t_pass in range(10):
        capi.sad_update_topk(prep, N, H, W, K, ma, mb, step_code(t_pass), J, 7)
        ma, mb = mb, ma
    state = {"t": t_pass + 1, "it": 0, "ma": ma, "mb": mb}

    def step(timed_parts=None):
        state["it"] += 1
        capi.sad_prepare_sites(pt, H, W, prep)
        if timed_parts is not None:
            timed_parts["u0"].record()
        capi.sad_update_topk(prep, N, H, W, K, state["ma"], state["mb"], step_code(state["t"]), J, 7)
        if timed_parts is not None:
            timed_parts["u1"].record()
        state["ma"], state["mb"] = state["mb"], state["ma"]
        state["t"] += 1
        capi.sad_train_grads(pt, prep, H, W, K, state["ma"], target, grads, loss, ws)
        if timed_parts is not None:
            timed_parts["g1"].record()
        capi.sad_adam_step(pt, grads, m, v, H, W, state["it"], hp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st, used = capi.sad_workspace_status(ws)
    if st != 0:
        raise RuntimeError(f"workspace overflow during warm-up ({used} records)")

    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    evs = [{"s": E(), "u0": E(), "u1": E(), "g1": E(), "e": E()} for _ in range(args.steps)]
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.zero_()
        evs[i]["s"].record()
        step(evs[i])
        evs[i]["e"].record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    step_ms = [e["s"].elapsed_time(e["e"]) for e in evs]
    upd_ms = [e["u0"].elapsed_time(e["u1"]) for e in evs]
    grad_ms = [e["u1"].elapsed_time(e["g1"]) for e in evs]
    total_ms = sum(step_ms)
    if world > 1:
        tt = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    value = world * P * args.steps / (total_ms / 1e3) / 1e6

    # end to end through the public C-ABI binding with host buffers
    host_img = torch.from_numpy(img).pin_memory()
    host_loss = torch.empty(1, dtype=torch.float32).pin_memory()
    e2e_s = 0.0
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        target.copy_(host_img, non_blocking=True)
        step()
        host_loss.copy_(loss, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    e2e = {"value": world * P * args.steps / e2e_s / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": int(host_img.numel() * 4), "d2h_bytes_per_step": 4}

    peak, peak_kind = measured_peaks()
    g_ms = statistics.mean(grad_ms)
    alg_bytes = P * (K * 4 + 12) + N * (48 + 44)
    achieved = alg_bytes / (g_ms / 1e3) / 1e9
    roofline = {"kernel": "sad_train_grads (fused render+MSE+adjoint+segmented reduce)",
                "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind, "traffic": None,
                "algorithmic_bytes": alg_bytes, "avg_ms": round(g_ms, 5)}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "sites": N, "K": K, "J": J,
                   "l2": "flushed (256 MB write) before every timed step", "parallelism": f"replicas x{world}"},
        "breakdown_ms": {"update_topk": round(statistics.mean(upd_ms), 5),
                         "train_grads": round(g_ms, 5),
                         "prepare+adam": round(statistics.mean(step_ms) - statistics.mean(upd_ms) - g_ms, 5)},
        "encode_images_per_s_2000it": round(1e3 / (2000 * statistics.mean(step_ms)), 4),
        "e2e": e2e, "roofline": roofline, "clocks": ck,
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
    }
    if not args.no_c3:
        line["c3_render_backward"] = c3_leg(capi, dev, peak, peak_kind)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def c3_leg(capi, dev, peak, peak_kind, iters=10):
    """render + render_backward at 2048^2, 262144 random anisotropic sites, K=16."""
    import torch
    from paper_2604_21984_gb300 import inputs as gen
    H = W = 2048
    N, K = 262144, 16
    p = gen.sites_random_spd(H, W, N, seed=3000)
    pt = torch.from_numpy(p).to(dev)
    prep = capi.empty_prep(N, dev)
    capi.sad_prepare_sites(pt, H, W, prep)
    a, b = capi.empty_map(H, W, K, dev), capi.empty_map(H, W, K, dev)
    capi.sad_topk_seed(prep, N, H, W, K, a)
    for t in range(16):
        s = max(1, 2048 >> (min(t, 10) + 1))
        capi.sad_update_topk(prep, N, H, W, K, a, b, (s << 16) | t, 2, 11)
        a, b = b, a
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    g = torch.from_numpy(gen.grad_image(H, W, seed=3002) / (H * W)).to(dev)
    grads = torch.empty((11, N), dtype=torch.float32, device=dev)
    ws = capi.backward_workspace(H, W, K, N, device=dev)
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    for _ in range(3):
        capi.sad_render(prep, N, H, W, K, a, rgb)
        capi.sad_render_backward(pt, prep, H, W, K, a, g, grads, ws)
    torch.cuda.synchronize()
    st, used = capi.sad_workspace_status(ws)
    r_ms, b_ms = [], []
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
    P = H * W
    rb = statistics.mean(r_ms)
    bb = statistics.mean(b_ms)
    render_bytes = P * (K * 4 + 12) + N * 48
    bwd_bytes = P * (K * 4 + 12) + N * (48 + 44)
    return {
        "workload": "2048x2048, 262144 random anisotropic sites, K=16, map from seed + 16 passes",
        "mpix_per_s_fwd_bwd": round(P / ((rb + bb) / 1e3) / 1e6, 1),
        "render_ms": round(rb, 4), "backward_ms": round(bb, 4), "records": used, "ws_status": st,
        "roofline_render": {"bound": "hbm", "achieved": round(render_bytes / (rb / 1e3) / 1e9, 1),
                            "peak": peak, "unit": "GB/s",
                            "frac": round(render_bytes / (rb / 1e3) / 1e9 / peak, 4), "peak_kind": peak_kind},
        "roofline_fwd_bwd": {"bound": "hbm",
                             "achieved": round((render_bytes + bwd_bytes) / ((rb + bb) / 1e3) / 1e9, 1),
                             "peak": peak, "unit": "GB/s",
                             "frac": round((render_bytes + bwd_bytes) / ((rb + bb) / 1e3) / 1e9 / peak, 4),
                             "peak_kind": peak_kind},
    }


# ----------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline key)
# ----------------------------------------------------------------------------

CPU_CROP = 128


def _cpu_sample():
    """A CROPxCROP window of the workload image with the sites inside it (same
    density), K=16, J=4, field warmed up by seed + 8 passes (untimed)."""
    import numpy as np
    from oracle import sad_oracle as oracle
    img, params = c2_inputs(0)
    c = CPU_CROP
    sub = img[:c, :c].copy()
    inside = (params[0] < c) & (params[1] < c)
    p = params[:, inside].copy()
    ids = oracle.propagate_fp32(p, c, c, K_C2, passes=8, J=J_C2, seed=7)
    return oracle, np, sub, p, ids


def _cpu_iteration(oracle, np, sub, p, ids, t, m, v):
    c = CPU_CROP
    prep = oracle.prepare_fp32(p, c, c)
    ids = oracle.topk_pass_fp32(prep, ids, c, c, K_C2, (1 << 16) | (t & 0xFFFF), J_C2, 7)
    rgb = oracle.render(p, c, c, ids)
    _, g = oracle.mse_loss_and_grad_rgb(rgb, sub)
    grads = oracle.render_backward(p, c, c, ids, g)
    p2, m, v = oracle.adam_step(p, grads, m, v, t, c, c)
    return p2.astype(np.float32), ids, m, v


def cpu_baseline(budget_s=12.0):
    oracle, np, sub, p, ids = _cpu_sample()
    m = np.zeros(p.shape)
    v = np.zeros(p.shape)
    n, t0 = 0, time.perf_counter()
    while True:
        p, ids, m, v = _cpu_iteration(oracle, np, sub, p, ids, n + 1, m, v)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 50:
            break
    return {"value": round(CPU_CROP * CPU_CROP * n / el / 1e6, 5), "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": f"{n} training iterations on a {CPU_CROP}x{CPU_CROP} crop of the workload image "
                      f"(sites inside it, K=16, J=4), numpy single-threaded, {el:.1f} s"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    oracle, np, sub, p, ids = _cpu_sample()
    m = np.zeros(p.shape)
    v = np.zeros(p.shape)
    for i in range(args.warmup):
        p, ids, m, v = _cpu_iteration(oracle, np, sub, p, ids, i + 1, m, v)
    t0 = time.perf_counter()
    for i in range(args.steps):
        p, ids, m, v = _cpu_iteration(oracle, np, sub, p, ids, args.warmup + i + 1, m, v)
    el = time.perf_counter() - t0
    value = CPU_CROP * CPU_CROP * args.steps / el / 1e6
    sample = (f"{args.steps} timed training iterations on a {CPU_CROP}x{CPU_CROP} crop of the "
              f"workload image, numpy single-threaded")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el * 1e3 / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H_C2, "W": W_C2, "sites": N_C2, "K": K_C2, "J": J_C2,
                   "parallelism": "cpu oracle"},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
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
