#!/usr/bin/env python3
"""Throughput benchmark: Mrays/s of forward + PRB adjoint on one GB300 (per rank).

Workload (the forward-throughput configuration): 32 noise-displaced level-4
icospheres (5,120 triangles each) on a 128x128-quad ground plane (196,608
triangles), textured diffuse / GGX conductor / dielectric, 512x256 sky
environment map, 1024x1024 pixels, 64 spp, max depth 8, Russian roulette from
depth 3.  One step = one forward render (megakernel) + one adjoint render (path
replay backpropagation, decorrelated seed) with the L2-loss image gradient
against a fixed target, gradients into the 1024^2 RGBA texture and the
conductor roughness values.  Rays = closest-hit + shadow rays, counted by an
instrumented launch of the same step before timing.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s fwd+adjoint on 1 GB300 vs roofline; equal-time MSE, cache vs plain PT"
WORKLOAD = dict(workload="spheres32x5120 + ground 128^2 (196,608 tris), 1024x1024, 64 spp, depth 8, RR from 3, "
                         "forward + PRB adjoint (texture 1024^2 RGBA + roughness gradients)",
                width=1024, height=1024, spp=64, max_depth=8, rr_depth=3)
FLOPS_PER_NODE = {"binary": 44,   # two child slab tests: 12 FMA (24 flops), 10 min/max, 2 compares, ordering
                  "wide": 140}    # eight child slab tests: 48 FMA (96 flops), 40 min/max, 8 compares (per-node
                                  # decode: 3 scale + 3 offset products excluded)
FLOPS_PER_TRI = 45      # Moller-Trumbore: 2 cross, 4 dot, 1 div, 4 mul, 3 sub (FMA = 2 flops)
NODE_BYTES = {"binary": 64, "wide": 80}  # bytes fetched per node visit
TRI_BYTES, TEX_BYTES, ENV_BYTES = 48, 16, 16  # per triangle test, texture lookup, env-map lookup
# FP32 operations per shaded vertex (FMA = 2), counted from the kernel's per-vertex
# formulas: hit point, barycentric uv, geometric normal, frame and local directions
# (~85 for every type); the light sample, BSDF value and pdf toward it, MIS weight and
# shadow-ray offset (none at a smooth dielectric); the BSDF sample with its value and
# pdf, the throughput update and the continuation-ray offset.  GGX adds the half
# vector, D, two Smith G1 and three Schlick terms to every evaluation.
SHADE_FLOPS = {8: 250, 9: 415, 10: 130, 11: 450}   # counter index -> diffuse, conductor, dielectric, blend
ENV_FLOPS = 60          # direction -> env pixel (atan2, acos), its pdf and the MIS weight
GRAD_BYTES_TEX, GRAD_BYTES_OTHER = 16, 4  # one float4 texel / one float per gradient term (before aggregation)


def counted_work(c, bvh):
    """(FP32 flops, bytes through L2) of the counted work c (PT_CNT_* array)."""
    c = [int(x) for x in c]
    flops = (FLOPS_PER_NODE[bvh] * c[3] + FLOPS_PER_TRI * c[4] + sum(v * c[k] for k, v in SHADE_FLOPS.items())
             + ENV_FLOPS * c[12])
    nbytes = NODE_BYTES[bvh] * c[3] + TRI_BYTES * c[4] + TEX_BYTES * c[5] + ENV_BYTES * c[12]
    grad_bytes = GRAD_BYTES_TEX * c[13] + GRAD_BYTES_OTHER * (c[7] - c[13])
    return flops, nbytes, grad_bytes


def alu_roofline(kernel, counters, bvh, ms, clk, note=""):
    """FP32-ALU roofline entry: traversal FLOPs of the counted node visits and
    triangle tests (counters = PT_CNT_* array) over `ms`, against 152 SMs x 128 lanes
    x 2 x the median SM clock sampled during the timed region."""
    import torch
    flops = FLOPS_PER_NODE[bvh] * int(counters[3]) + FLOPS_PER_TRI * int(counters[4])
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or 1477.0
    peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    achieved = flops / (ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": round(achieved, 3), "peak": round(peak, 2),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
            "work": f"{FLOPS_PER_NODE[bvh]}/node visit + {FLOPS_PER_TRI}/triangle test (counted launch){note}",
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x median SM clock {mhz} MHz"}
# DRAM bytes (read + write) per counted ray of a production kernel, from a one-kernel,
# few-launch ncu capture of the 256x256 case (profiles/), scaled to a full-size launch
# by its counted rays (the per-ray traffic of these kernels does not depend on the
# image size: the scene and texture are the same and the per-sample state scales with
# the rays).  A kernel changed since its capture has no entry.
TRAFFIC_PER_RAY = {"wide": {"forward_kernel": 52.2, "radiance_kernel": 71.0, "replay_kernel": 146.5}}
# reparam_kernel (translation mode): DRAM bytes per sample of the same kind of capture
# (409 MB per 256x256 x 4 spp launch).
REPARAM_TRAFFIC_PER_SAMPLE = 1535.0
TRAFFIC_BASIS = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per counted ray at 256x256 "
                 "(profiles/dram_per_ray_spheres196k_256px_64spp.md), times the launch's counted rays")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cache-line", action="store_true",
                    help="skip the equal-time cache-vs-plain comparison of the default line")
    ap.add_argument("--dispatch", type=int, default=0)
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--tex-aggregate", type=int, default=0)
    ap.add_argument("--prb-mode", type=int, default=0, help="backward: 0 auto (split), 1 fused PRB, 2 split")
    ap.add_argument("--bvh", default="wide", choices=["wide", "binary"])
    ap.add_argument("--schedule", type=int, default=0,
                    help="0 auto (= static), 1 persistent lanes pulling units, 2 static: one unit per thread")
    ap.add_argument("--cache", action="store_true",
                    help="radiance-cache experiment: equal-time MSE, cache-terminated vs plain PT (own JSON line)")
    ap.add_argument("--cache-warmup-frames", type=int, default=300)
    ap.add_argument("--cache-ema", type=float, default=0.99, help="moving average of the cache weights (0 = off)")
    ap.add_argument("--batch", action="store_true",
                    help="batching experiment: 64 cameras over 10k/200k/2M-triangle scenes, forward + adjoint "
                         "in one persistent graph-captured launch vs 64 separate launches (own JSON line)")
    ap.add_argument("--jvp", action="store_true",
                    help="forward-mode image derivative on the throughput workload vs the plain forward (own line)")
    ap.add_argument("--wavefront", action="store_true",
                    help="megakernel vs wavefront ablation, forward and adjoint (own JSON line)")
    ap.add_argument("--wave-paths", type=int, default=0)
    ap.add_argument("--mlp", action="store_true",
                    help="radiance-cache MLP inference throughput, tcgen05 vs mma.sync engines (own JSON line)")
    ap.add_argument("--ckpt", action="store_true",
                    help="PRB vs reverse mode with checkpoints, one gradient step each (own JSON line)")
    ap.add_argument("--trace", action="store_true",
                    help="ray queries alone (pt_trace_rays) on the sphere scene: coherent camera rays and "
                         "incoherent surface rays, closest and any hit, G rays/s (own JSON line)")
    ap.add_argument("--texgrad", action="store_true",
                    help="PRB adjoint of the 96-shape textured room (2048^2 atlas + 96 roughness values): "
                         "Mrays/s and gradient atomics/s (own JSON line)")
    ap.add_argument("--reparam", action="store_true",
                    help="reparameterized PRB: shape-translation gradients through visibility (own JSON line)")
    ap.add_argument("--reparam-spp", type=int, default=16)
    ap.add_argument("--peaks", action="store_true",
                    help="microbenchmarks of the memory-side roofs (L2-resident reads, atomics) as a JSON line")
    ap.add_argument("--small", action="store_true",
                    help="profiling case: same scene and step at 256x256, 64 spp (not a bench line)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workload
def make_workload(seed=2022, small=False):
    from paper_2202_01284_gb300 import scenes as S
    sc = S.spheres(seed, width=256, height=256) if small else S.spheres(seed)
    tgt_tex = S.spheres_target_texture(sc.textures[0], seed)
    return sc, tgt_tex


def settings(args, seed):
    from paper_2202_01284_gb300.render import RenderSettings
    if args.small:
        return RenderSettings(width=256, height=256, spp=64, max_depth=WORKLOAD["max_depth"],
                              rr_depth=WORKLOAD["rr_depth"], seed=seed, dispatch=args.dispatch,
                              lanes_per_pixel=args.lanes, block_size=args.block, tex_aggregate=args.tex_aggregate,
                              prb_mode=args.prb_mode, schedule=args.schedule)
    return RenderSettings(width=WORKLOAD["width"], height=WORKLOAD["height"], spp=WORKLOAD["spp"],
                          max_depth=WORKLOAD["max_depth"], rr_depth=WORKLOAD["rr_depth"], seed=seed,
                          dispatch=args.dispatch, lanes_per_pixel=args.lanes, block_size=args.block,
                          tex_aggregate=args.tex_aggregate, prb_mode=args.prb_mode, schedule=args.schedule)


# Bounded samples of the workload for the FP64 oracle on the host cores: the
# CPU-baseline leg of our arm (~10 s on 16 Grace cores) and one step of the
# reference arm (~3 s, so that --steps 5 --warmup 3 stays well under a minute).
CPU_BASELINE_CROP = (256, 320, 512, 384)
REFERENCE_STEP_CROP = (384, 384, 256, 256)


def cpu_baseline_run(sc, steps=1, crop=CPU_BASELINE_CROP):
    """The FP64 oracle as it stands on the host cores, on a bounded crop of the workload."""
    import numpy as np
    import oracle
    osc = oracle.OracleScene(sc)
    cam = sc.cameras[0]
    spp = 64
    r = oracle.render_in(cam, spp, WORKLOAD["max_depth"], 11, WORKLOAD["rr_depth"], True, crop=crop)
    cores = os.cpu_count() or 1
    vals = []
    total_rays = 0
    for _ in range(steps):
        t0 = time.perf_counter()
        img, rays_f = oracle.render(osc, r, threads=cores, count_rays=True)
        gi = 2 * (img - 0.5) / img.size
        *_, rays_b = oracle.grad_tape(osc, r, gi, threads=cores, count_rays=True)
        dt = time.perf_counter() - t0
        vals.append((rays_f + rays_b) / dt / 1e6)
        total_rays += rays_f + rays_b
    return {"value": statistics.median(vals), "unit": "Mrays/s", "cores": cores, "kind": "oracle",
            "sample": f"{crop[2]}x{crop[3]} pixel crop at ({crop[0]},{crop[1]}), {spp} spp, depth 8, RR 3: "
                      f"FP64 render + stored-tape adjoint, {total_rays} rays"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc, _ = make_workload()
    steps = max(1, args.steps)
    for _ in range(max(0, args.warmup)):
        cpu_baseline_run(sc, steps=1, crop=REFERENCE_STEP_CROP)
    cb = cpu_baseline_run(sc, steps=steps, crop=REFERENCE_STEP_CROP)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "Mrays/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**WORKLOAD, "sample": cb["sample"]},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2202_01284_gb300 import abi
    from paper_2202_01284_gb300.render import DeviceScene

    from paper_2202_01284_gb300 import dist as D

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    abi.load()

    sc, tgt_tex = make_workload(small=args.small)
    layout = abi.PT_BVH_WIDE if args.bvh == "wide" else abi.PT_BVH_BINARY
    ds = DeviceScene(sc, layout=layout, device=dev)
    seed_fwd, seed_bwd = D.rank_seeds(rank)  # replicas: every rank renders its own samples
    st_f = settings(args, seed_fwd)
    # fixed target image (rendered once) -> dLoss/dImage for the adjoint
    target = ds.forward(settings(args, 77), textures=[torch.as_tensor(tgt_tex, device=dev)]).clone()
    img = torch.empty_like(target)
    g_tex = torch.zeros_like(ds.textures[0])
    g_rough = torch.zeros_like(ds.roughness)
    grad_img = torch.empty_like(target)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        ds.forward(st_f, out=img)
        if ev is not None:
            ev[1].record(stream)
        torch.sub(img, target, out=grad_img)
        grad_img.mul_(2.0 / img.numel())
        if ev is not None:
            ev[2].record(stream)
        ds.backward(st_f, grad_img, g_textures=[g_tex], g_roughness=g_rough, seed=seed_bwd)
        if ev is not None:
            ev[3].record(stream)

    # ray counts of one step (instrumented launches of the identical work)
    cf = torch.zeros(abi.PT_N_COUNTERS, dtype=torch.int64, device=dev)
    cb = torch.zeros(abi.PT_N_COUNTERS, dtype=torch.int64, device=dev)
    ds.forward(st_f, out=img, counters=cf)
    torch.sub(img, target, out=grad_img)
    grad_img.mul_(2.0 / img.numel())
    ds.backward(st_f, grad_img, g_textures=[torch.zeros_like(g_tex)], g_roughness=torch.zeros_like(g_rough),
                seed=seed_bwd, counters=cb)
    torch.cuda.synchronize()
    cf, cb = cf.cpu().numpy(), cb.cpu().numpy()
    rays_f = int(cf[1] + cf[2])
    rays_b = int(cb[1] + cb[2])
    rays_step = rays_f + rays_b
    flops_f, bytes_f, _ = counted_work(cf, args.bvh)
    flops_b, bytes_b, grad_bytes_b = counted_work(cb, args.bvh)
    # memory-side roofs with the library's own probes (before the timed region)
    roofs = measure_roofs(torch, dev)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))       # evict L2 between timed steps (outside the events)
        step(evs[k])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    fwd_ms = [e[0].elapsed_time(e[1]) for e in evs]
    adj_ms = [e[2].elapsed_time(e[3]) for e in evs]
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    total_ms = D.max_over_ranks(sum(step_ms), device=dev)
    value = rays_step * args.steps * world / (total_ms / 1e3) / 1e6

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    h_tex = torch.as_tensor(sc.textures[0]).pin_memory()
    h_rough = torch.as_tensor(sc.roughness).pin_memory()
    h_img = torch.empty(img.shape, dtype=torch.float32).pin_memory()
    h_gtex = torch.empty(g_tex.shape, dtype=torch.float32).pin_memory()
    h_grough = torch.empty(g_rough.shape, dtype=torch.float32).pin_memory()
    d_tex = torch.empty_like(ds.textures[0])
    d_rough = torch.empty_like(ds.roughness)

    def e2e_step():
        d_tex.copy_(h_tex, non_blocking=True)
        d_rough.copy_(h_rough, non_blocking=True)
        ds.forward(st_f, out=img, textures=[d_tex], roughness=d_rough)
        torch.sub(img, target, out=grad_img)
        grad_img.mul_(2.0 / img.numel())
        g_tex.zero_()
        g_rough.zero_()
        ds.backward(st_f, grad_img, textures=[d_tex], roughness=d_rough, g_textures=[g_tex], g_roughness=g_rough,
                    seed=seed_bwd)
        h_img.copy_(img, non_blocking=True)
        h_gtex.copy_(g_tex, non_blocking=True)
        h_grough.copy_(g_rough, non_blocking=True)
    e2e_step()
    torch.cuda.synchronize()
    # host wall clock around each call sequence, through the synchronisation that makes
    # the results readable on the host (L2 flushed before each step, outside the clock)
    e_steps = max(2, min(args.steps, 5))
    e_times = []
    for k in range(e_steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e_times.append(time.perf_counter() - t_a)
    e2e_ms = 1e3 * statistics.mean(e_times)
    h2d = h_tex.numel() * 4 + h_rough.numel() * 4
    d2h = h_img.numel() * 4 + h_gtex.numel() * 4 + h_grough.numel() * 4

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    fwd_avg, adj_avg = statistics.mean(fwd_ms), statistics.mean(adj_ms)
    split = args.prb_mode != abi.PT_PRB_FUSED
    if split:
        # the adjoint stage is a radiance pass (the forward megakernel with the adjoint
        # seed, storing each sample's L) + the replay kernel: time that radiance pass
        # on its own (after the timed region) to attribute the stage to its kernels
        from dataclasses import replace
        st_r = replace(st_f, seed=seed_bwd)
        ev_r = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(float(k))
            ev_r[k][0].record(stream)
            ds.forward(st_r, out=img)
            ev_r[k][1].record(stream)
        torch.cuda.synchronize()
        rad_avg = statistics.mean(a.elapsed_time(b) for a, b in ev_r)
        replay_avg = adj_avg - rad_avg
        # the replay runs as the persistent instance unless a static schedule was asked for
        kern = {"forward_kernel": (fwd_avg, flops_f), "replay_kernel": (replay_avg, flops_b / 2)}
        replay_name = "replay_persist_kernel" if args.schedule == 1 else "replay_kernel"
    else:
        rad_avg = replay_avg = None
        kern = {"forward_kernel": (fwd_avg, flops_f), "adjoint_kernel": (adj_avg, flops_b)}
        replay_name = None
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms, dom_flops = kern[dom]
    # the same kernel's bytes through L2: node, triangle, texel and env fetches of the
    # counted work, plus (replay / adjoint) the gradient scatter before aggregation
    dom_bytes = {"forward_kernel": bytes_f, "replay_kernel": bytes_b / 2 + grad_bytes_b,
                 "adjoint_kernel": bytes_b + grad_bytes_b}[dom]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 1477.0
    peak_tflops = sms * 128 * 2 * mhz * 1e6 / 1e12
    achieved = dom_flops / (dom_ms / 1e3) / 1e12
    achieved_gbs = dom_bytes / (dom_ms / 1e3) / 1e9
    alu_frac = achieved / peak_tflops
    l2_frac = achieved_gbs / roofs["l2_read_gbs"]
    traffic = (TRAFFIC_PER_RAY.get(args.bvh, {}).get(dom, 0) * {"forward_kernel": rays_f, "replay_kernel": rays_b / 2,
               "adjoint_kernel": rays_b}[dom]) or None
    if l2_frac >= alu_frac:
        head = {"bound": "l2", "achieved": round(achieved_gbs, 1), "peak": roofs["l2_read_gbs"], "unit": "GB/s",
                "frac": round(l2_frac, 4)}
    else:
        head = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_tflops, 2), "unit": "TFLOP/s",
                "frac": round(alu_frac, 4)}
    kernel_name = replay_name if dom == "replay_kernel" else dom
    traffic = (TRAFFIC_PER_RAY.get(args.bvh, {}).get(kernel_name, 0) * {"forward_kernel": rays_f,
               "replay_kernel": rays_b / 2, "adjoint_kernel": rays_b}[dom]) or None
    roofline = {**head, "kernel": kernel_name, "traffic": round(traffic) if traffic else None,
                "traffic_basis": TRAFFIC_BASIS if traffic else "no capture of the current kernel",
                "alu": {"achieved_tflops": round(achieved, 3), "peak_tflops": round(peak_tflops, 2),
                        "frac": round(alu_frac, 4),
                        "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x median SM clock {mhz} MHz",
                        "work": f"{FLOPS_PER_NODE[args.bvh]}/node visit + {FLOPS_PER_TRI}/triangle test + "
                                "shading per vertex (diffuse 250, conductor 415, dielectric 130, blend 450, "
                                f"env lookup {ENV_FLOPS}), counted launch"},
                "l2": {"achieved_gbs": round(achieved_gbs, 1), "peak_gbs": roofs["l2_read_gbs"],
                       "frac": round(l2_frac, 4),
                       "bytes": f"{NODE_BYTES[args.bvh]} B/node visit + {TRI_BYTES} B/triangle test + "
                                f"{TEX_BYTES} B/texel + {ENV_BYTES} B/env lookup"
                                + (" + 16 B/texel gradient term + 4 B/other term" if dom != "forward_kernel" else ""),
                       "peak_basis": "pt_probe_read, L2-resident 16-B loads, measured in this run"},
                "timing": ("replay = half of the counted fused adjoint; its time = adjoint stage minus the radiance "
                           "pass timed alone" if dom == "replay_kernel" else "CUDA events around the launch")}
    if dom != "forward_kernel":
        terms = int(cb[7])
        roofline["atomics"] = {"grad_terms_per_s_g": round(terms / (dom_ms / 1e3) / 1e9, 3),
                               "issued_after_aggregation": int(cb[6]),
                               "peak_f4_spread_gops": roofs["red_f4_spread_1M_gops"],
                               "peak_f1_colliding_96_gops": roofs["red_f1_colliding_96_gops"]}
    cache_line = None
    if not args.no_cache_line and not args.small and world == 1:
        try:
            cc = cache_comparison(torch, warmup_frames=300, spps=(64, 96, 128, 192, 256, 320))
            cache_line = {"workload": cc["workload"], "reference_spp": cc["reference_spp"],
                          "plain": cc["plain"], "indirect_pixel_fraction": cc["indirect_pixel_fraction"]}
            for k in ("cache_bounce1", "cache_bounce2"):
                c = cc[k]
                cache_line[k] = {kk: c[kk] for kk in ("equal_time_spp", "equal_time", "train_loss",
                                                      "mse_indirect_ratio_plain_over_cache",
                                                      "mse_ratio_plain_over_cache", "warmup_frames",
                                                      "weight_average")}
        except Exception as e:  # the throughput line stands without it
            cache_line = {"error": str(e)[:300]}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = cpu_baseline_run(sc)
        except Exception as e:  # the oracle is optional for the GPU number
            cpu = {"error": str(e)}
    info = ds.info()
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**WORKLOAD, "l2": "flushed between timed steps (256 MB write)", "dispatch": args.dispatch,
                   "schedule": ["auto: one unit per thread", "persistent lanes", "static: one unit per thread"][
                       args.schedule],
                   "bvh": f"{args.bvh} SAH", "bvh_nodes": info["n_nodes"], "rays_per_step": rays_step,
                   "rays_fwd": rays_f, "rays_adj": rays_b, "fwd_ms": round(fwd_avg, 3),
                   "adj_ms": round(adj_avg, 3), "prb": "split" if split else "fused",
                   "adj_radiance_pass_ms": round(rad_avg, 3) if split else None,
                   "adj_replay_ms": round(replay_avg, 3) if split else None,
                   "fwd_mrays_s": round(rays_f / fwd_avg / 1e3, 1),
                   "adj_mrays_s": round(rays_b / adj_avg / 1e3, 1),
                   "node_visits_per_ray_fwd": round(int(cf[3]) / max(rays_f, 1), 2),
                   "tri_tests_per_ray_fwd": round(int(cf[4]) / max(rays_f, 1), 2),
                   "grad_terms": int(cb[7]), "grad_atomics": int(cb[6]),
                   "paths_per_step": int(cf[0] + cb[0]) // (2 if split else 1),
                   "mpaths_s_fwd": round(int(cf[0]) / fwd_avg / 1e3, 1),
                   "shaded_vertices_fwd": {"diffuse": int(cf[8]), "conductor": int(cf[9]), "dielectric": int(cf[10]),
                                           "blend": int(cf[11])},
                   "env_lookups_fwd": int(cf[12]),
                   "simt": {"traversal_lanes_per_node_step_fwd": round(32 * int(cf[3]) / max(32 * int(cf[14]), 1), 2),
                            "rays_per_loop_step_fwd": round(32 * int(cf[1] + cf[2]) / max(32 * int(cf[15]), 1), 2),
                            "traversal_lanes_per_node_step_adj": round(32 * int(cb[3]) / max(32 * int(cb[14]), 1), 2),
                            "rays_per_loop_step_adj": round(32 * int(cb[1] + cb[2]) / max(32 * int(cb[15]), 1), 2),
                            "basis": "counted launch: lanes per warp-level iteration (of 32)"},
                   "measured_roofs": roofs},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cache_vs_plain": cache_line,
        "e2e": {"value": round(rays_step / (e2e_ms / 1e3) / 1e6, 2), "unit": "Mrays/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3),
                "timing": "host wall clock per step through the C ABI calls and the final synchronisation; "
                          "pinned host inputs copied in, image and gradients copied out"},
        "gpu_launches": (3 if split else 2) * args.steps,
        "clocks": clk,
        "wall_s": round(wall, 3),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_trace_experiment(args):
    """Ray queries alone, through the megakernels' traversal (pt_trace_rays), on the
    sphere scene's 8-wide BVH: 2048^2 jittered camera rays (coherent) and as many rays
    leaving random surface points in uniform hemisphere directions (incoherent, like
    the path tracer's bounces), closest hit, and the incoherent set again as any-hit
    queries without a distance limit.  Rays are made on the device from a seeded
    torch generator; 100 MB of rays per set, the L2 flushed before every launch.  The
    megakernel's rays/s include shading and sampling; these are the traversal's.
    Own JSON line."""
    import math

    import torch

    from paper_2202_01284_gb300 import abi
    from paper_2202_01284_gb300 import scenes as S
    from paper_2202_01284_gb300.render import DeviceScene
    abi.load()
    dev = torch.device("cuda", 0)
    sc = S.spheres()
    ds = DeviceScene(sc, layout=abi.PT_BVH_WIDE, device=dev)
    w = 512 if args.small else 2048
    n = w * w
    g = torch.Generator(device=dev).manual_seed(2022)
    cam = sc.cameras[0]
    o = torch.tensor(cam.origin, dtype=torch.float32, device=dev)
    f = torch.tensor(cam.target, dtype=torch.float32, device=dev) - o
    f = f / f.norm()
    r = torch.linalg.cross(f, torch.tensor(cam.up, dtype=torch.float32, device=dev))
    r = r / r.norm()
    u = torch.linalg.cross(r, f)
    th = math.tan(math.radians(cam.vfov_deg) / 2)
    iy, ix = torch.meshgrid(torch.arange(w, device=dev), torch.arange(w, device=dev), indexing="ij")
    jit = torch.rand((w, w, 2), device=dev, generator=g)
    sx = (2 * (ix + jit[..., 0]) / w - 1).reshape(-1, 1) * th * cam.width / cam.height
    sy = (1 - 2 * (iy + jit[..., 1]) / w).reshape(-1, 1) * th
    d = f + sx * r + sy * u
    cam_rays = torch.cat([o.expand(n, 3), d / d.norm(dim=1, keepdim=True)], 1).contiguous()
    V = torch.as_tensor(sc.vertices, dtype=torch.float32, device=dev)
    ti = torch.randint(0, V.shape[0], (n,), device=dev, generator=g)
    b = -torch.log(torch.rand((n, 3), device=dev, generator=g).clamp_min(1e-12))  # rand may return 0
    b = b / b.sum(1, keepdim=True)
    p = (b[:, :, None] * V[ti]).sum(1)
    nrm = torch.linalg.cross(V[ti, 1] - V[ti, 0], V[ti, 2] - V[ti, 0])
    nrm = nrm / nrm.norm(dim=1, keepdim=True).clamp_min(1e-30)
    dd = torch.randn((n, 3), device=dev, generator=g)
    dd = dd / dd.norm(dim=1, keepdim=True)
    dd = torch.where((dd * nrm).sum(1, keepdim=True) < 0, -dd, dd)
    eps = 1e-4 * max(1.0, float(V.abs().max()))
    sec_rays = torch.cat([p + eps * nrm, dd], 1).contiguous()
    t = torch.empty(n, device=dev)
    prim = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    clocks = ClockSampler(0)
    clocks.start()
    for name, rays, any_hit in (("camera_closest", cam_rays, False), ("surface_closest", sec_rays, False),
                                ("surface_any", sec_rays, True)):
        for _ in range(max(3, args.warmup)):
            abi.pt_trace_rays(ds.handle, rays, n, t, prim, any_hit=any_hit, stream=stream.cuda_stream)
        ms = []
        for k in range(args.steps):
            flush.fill_(float(k))
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            abi.pt_trace_rays(ds.handle, rays, n, t, prim, any_hit=any_hit, stream=stream.cuda_stream)
            e.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(e))
        hit = float((prim >= 0).float().mean())
        res[name] = {"ms": round(statistics.mean(ms), 4), "grays_s": round(n / statistics.mean(ms) / 1e6, 3),
                     "hit_fraction": round(hit, 4)}
    clk = clocks.stop()
    assert ds.status() == 0
    line = {"metric": "ray queries through the path tracer's traversal, G rays/s (surface rays, closest hit)",
            "value": res["surface_closest"]["grays_s"], "unit": "G rays/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"spheres32x5120 + ground (196,608 tris), 8-wide BVH, {n} rays per set",
                       "l2": "flushed before each launch", "sets": res},
            "gpu_launches": 3 * args.steps, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_texgrad_experiment(args):
    """The texture-gradient configuration: the 96-shape Cornell room (blend BSDFs,
    one 2048^2 RGBA atlas texture, 96 roughness values), 512x512, 16 spp, depth 6, no
    roulette; one step = forward + PRB adjoint with the L2 gradient against the target
    texture's render.  Reports the adjoint's Mrays/s and the gradient atomics it
    issues per second (texel float4 and roughness atomics, before and after warp
    aggregation, counted by an instrumented launch).  Own JSON line."""
    import torch

    from paper_2202_01284_gb300 import abi
    from paper_2202_01284_gb300 import scenes as S
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    abi.load()
    dev = torch.device("cuda", 0)
    sc = S.cornell96(width=512, height=512)
    ds = DeviceScene(sc, layout=abi.PT_BVH_WIDE if args.bvh == "wide" else abi.PT_BVH_BINARY, device=dev)
    st = RenderSettings(width=512, height=512, spp=16, max_depth=6, rr_depth=-1, seed=11)
    tgt = torch.as_tensor(S.cornell96_target_texture(sc.textures[0]), device=dev)
    target = ds.forward(RenderSettings(width=512, height=512, spp=16, max_depth=6, rr_depth=-1, seed=77),
                        textures=[tgt]).clone()
    img = torch.empty_like(target)
    gi = torch.empty_like(target)
    g_tex = torch.zeros_like(ds.textures[0])
    g_rough = torch.zeros_like(ds.roughness)
    cf = torch.zeros(abi.PT_N_COUNTERS, dtype=torch.int64, device=dev)
    cb = torch.zeros_like(cf)
    ds.forward(st, out=img, counters=cf)
    torch.sub(img, target, out=gi)
    gi.mul_(2.0 / img.numel())
    ds.backward(st, gi, g_textures=[g_tex], g_roughness=g_rough, seed=12, counters=cb)
    torch.cuda.synchronize()
    cf, cb = cf.cpu().numpy(), cb.cpu().numpy()
    rays_f, rays_b = int(cf[1] + cf[2]), int(cb[1] + cb[2])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev):
        ev[0].record(stream)
        ds.forward(st, out=img)
        torch.sub(img, target, out=gi)
        gi.mul_(2.0 / img.numel())
        ev[1].record(stream)
        ds.backward(st, gi, g_textures=[g_tex], g_roughness=g_rough, seed=12)
        ev[2].record(stream)

    dummy = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(max(3, args.warmup)):
        step(dummy)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    evs = []
    for k in range(args.steps):
        flush.fill_(float(k))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        step(ev)
        evs.append(ev)
    torch.cuda.synchronize()
    clk = clocks.stop()
    fwd_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    adj_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    line = {"metric": "PRB adjoint of the textured 96-shape room: Mrays/s and gradient atomics/s",
            "value": round(rays_b / adj_ms / 1e3, 2), "unit": "Mrays/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(fwd_ms + adj_ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "cornell96 (96 blend shapes, 2048^2 RGBA atlas, 96 roughness values), "
                                   "512x512, 16 spp, depth 6, no roulette; forward + PRB adjoint",
                       "l2": "flushed before each timed step", "forward_ms": round(fwd_ms, 3),
                       "adjoint_ms": round(adj_ms, 3), "rays_fwd": rays_f, "rays_adj": rays_b,
                       "fwd_mrays_s": round(rays_f / fwd_ms / 1e3, 1),
                       "gradient_terms": int(cb[7]), "gradient_atomics": int(cb[6]),
                       "gradient_terms_per_s_g": round(int(cb[7]) / adj_ms / 1e6, 3),
                       "gradient_atomics_per_s_g": round(int(cb[6]) / adj_ms / 1e6, 3)},
            "roofline": alu_roofline("replay_kernel (after radiance_kernel)", cb, args.bvh, adj_ms, clk,
                                     "; the adjoint's rays over radiance pass + replay"),
            "clocks": clk}
    print(json.dumps(line), flush=True)


def run_jvp_experiment(args):
    """Forward-mode image derivative on the throughput workload: one pt_render_jvp
    pass (image and d image / d eps along a direction over the 1024^2 texture and
    the roughness values) against the plain forward render with the same seed,
    i.e. the same rays.  Own JSON line."""
    import torch

    from paper_2202_01284_gb300 import abi
    from paper_2202_01284_gb300.render import DeviceScene
    abi.load()
    dev = torch.device("cuda", 0)
    sc, _ = make_workload(small=args.small)
    layout = abi.PT_BVH_WIDE if args.bvh == "wide" else abi.PT_BVH_BINARY
    ds = DeviceScene(sc, layout=layout, device=dev)
    st = settings(args, 11)
    g = torch.Generator(device=dev).manual_seed(5)
    v_tex = torch.rand(ds.textures[0].shape, device=dev, generator=g)
    v_tex[..., 3] = 0
    v_rough = torch.randn(ds.roughness.shape, device=dev, generator=g)
    img = torch.empty((1, st.height, st.width, 3), device=dev)
    cf = torch.zeros(abi.PT_N_COUNTERS, dtype=torch.int64, device=dev)
    ds.forward(st, out=img, counters=cf)
    torch.cuda.synchronize()
    cf = cf.cpu().numpy()
    rays = int(cf[1] + cf[2])
    flops = FLOPS_PER_NODE[args.bvh] * int(cf[3]) + FLOPS_PER_TRI * int(cf[4])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def jvp():
        return ds.jvp(st, t_textures=[v_tex], t_roughness=v_rough)
    for _ in range(max(3, args.warmup)):
        jvp()
        ds.forward(st, out=img)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        jvp()
        ev[k][1].record(stream)
        flush.fill_(float(k) + 0.5)
        ev[k][2].record(stream)
        ds.forward(st, out=img)
        ev[k][3].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    jvp_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    fwd_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 1477.0
    peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    achieved = flops / (jvp_ms / 1e3) / 1e12
    line = {"metric": "Mrays/s of the forward-mode image derivative (image + JVP along a parameter direction)",
            "value": round(rays / jvp_ms / 1e3, 2), "unit": "Mrays/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(jvp_ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**WORKLOAD, "workload": "spheres32x5120 + ground 128^2 (196,608 tris), "
                       f"{st.width}x{st.height}, 64 spp, depth 8, RR from 3, image + JVP along a direction over "
                       "the texture and roughness",
                       "width": st.width, "height": st.height, "l2": "flushed before each timed launch",
                       "rays": rays, "jvp_ms": round(jvp_ms, 3), "forward_ms": round(fwd_ms, 3),
                       "jvp_over_forward": round(jvp_ms / fwd_ms, 3),
                       "forward_mrays_s": round(rays / fwd_ms / 1e3, 1)},
            "roofline": {"bound": "alu", "kernel": "jvp_kernel", "achieved": round(achieved, 3), "peak": round(peak, 2),
                         "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                         "traffic": None
                         if not args.small else None,
                         "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x median SM clock {mhz} MHz"},
            "gpu_launches": 2 * args.steps, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_wavefront_experiment(args):
    """Megakernel vs wavefront execution of the same estimator (forward and PRB
    adjoint) on the throughput workload: the wavefront variant in its two call
    modes (traced material switch, material-grouped shading kernels).  Own JSON line."""
    import torch

    from paper_2202_01284_gb300 import abi
    from paper_2202_01284_gb300.render import DeviceScene
    abi.load()
    dev = torch.device("cuda", 0)
    sc, tgt_tex = make_workload(small=args.small)
    layout = abi.PT_BVH_WIDE if args.bvh == "wide" else abi.PT_BVH_BINARY
    ds = DeviceScene(sc, layout=layout, device=dev)
    st = settings(args, 11)
    target = ds.forward(settings(args, 77), textures=[torch.as_tensor(tgt_tex, device=dev)]).clone()
    img = torch.empty_like(target)
    cf = torch.zeros(abi.PT_N_COUNTERS, dtype=torch.int64, device=dev)
    cb = torch.zeros(abi.PT_N_COUNTERS, dtype=torch.int64, device=dev)
    ds.forward(st, out=img, counters=cf)
    grad_img = (2.0 * (img - target) / img.numel()).contiguous()
    g_tex = torch.zeros_like(ds.textures[0])
    g_rough = torch.zeros_like(ds.roughness)
    ds.backward(st, grad_img, g_textures=[g_tex], g_roughness=g_rough, counters=cb)
    torch.cuda.synchronize()
    cf, cb = cf.cpu().numpy(), cb.cpu().numpy()
    rays_f, rays_b = int(cf[1] + cf[2]), int(cb[1] + cb[2])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    wave = args.wave_paths
    variants = {
        "megakernel_fwd": lambda: ds.forward(st, out=img),
        "wavefront_traced_fwd": lambda: ds.wavefront_forward(st, calls=abi.PT_WF_TRACED, wave_paths=wave, out=img),
        "wavefront_grouped_fwd": lambda: ds.wavefront_forward(st, calls=abi.PT_WF_GROUPED, wave_paths=wave, out=img),
        "megakernel_adj": lambda: ds.backward(st, grad_img, g_textures=[g_tex], g_roughness=g_rough),
        "wavefront_traced_adj": lambda: ds.wavefront_backward(st, grad_img, calls=abi.PT_WF_TRACED, wave_paths=wave,
                                                              g_textures=[g_tex], g_roughness=g_rough),
        "wavefront_grouped_adj": lambda: ds.wavefront_backward(st, grad_img, calls=abi.PT_WF_GROUPED,
                                                               wave_paths=wave, g_textures=[g_tex],
                                                               g_roughness=g_rough),
    }
    for fn in variants.values():
        for _ in range(max(3, args.warmup)):
            fn()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ms = {k: [] for k in variants}
    for k in range(args.steps):
        for name, fn in variants.items():
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ms[name].append((a, b))
    torch.cuda.synchronize()
    clk = clocks.stop()
    avg = {k: statistics.mean(a.elapsed_time(b) for a, b in v) for k, v in ms.items()}
    mr = {k: round((rays_f if k.endswith("fwd") else rays_b) / v / 1e3, 1) for k, v in avg.items()}
    # per-path state through HBM: 16-byte words of PathState per slot
    line = {"metric": "megakernel vs wavefront: ms and Mrays/s, forward and PRB adjoint",
            "value": round(avg["wavefront_traced_fwd"] / avg["megakernel_fwd"], 3),
            "unit": "x slowdown of the wavefront (traced calls) forward vs the megakernel forward",
            "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD["workload"] if not args.small else "spheres 256x256 64 spp",
                       "wave_paths": wave or 4 * 1024 * 1024, "l2": "flushed before each timed launch",
                       "rays_fwd": rays_f, "rays_adj": rays_b,
                       "ms": {k: round(v, 3) for k, v in avg.items()}, "mrays_s": mr,
                       "slowdown_vs_megakernel": {
                           "traced_fwd": round(avg["wavefront_traced_fwd"] / avg["megakernel_fwd"], 3),
                           "grouped_fwd": round(avg["wavefront_grouped_fwd"] / avg["megakernel_fwd"], 3),
                           "traced_adj": round(avg["wavefront_traced_adj"] / avg["megakernel_adj"], 3),
                           "grouped_adj": round(avg["wavefront_grouped_adj"] / avg["megakernel_adj"], 3)}},
            "roofline": alu_roofline("wavefront forward (wf_start, wf_trace, wf_shade, wf_finish, wf_film)", cf,
                                     args.bvh, avg["wavefront_traced_fwd"], clk,
                                     "; the megakernel forward's rays, whole wavefront forward time"),
            "clocks": clk}
    print(json.dumps(line), flush=True)


def run_ckpt_experiment(args):
    """PRB against reverse mode with checkpoints (one per path vertex) on the
    throughput workload: one gradient step each (forward image, L2-loss image
    gradient, reverse pass), plus the checkpoint memory.  Own JSON line."""
    import torch

    from paper_2202_01284_gb300 import abi
    from paper_2202_01284_gb300.render import Checkpoints, DeviceScene, ckpt_backward, ckpt_forward
    abi.load()
    dev = torch.device("cuda", 0)
    sc, tgt_tex = make_workload(small=args.small)
    layout = abi.PT_BVH_WIDE if args.bvh == "wide" else abi.PT_BVH_BINARY
    ds = DeviceScene(sc, layout=layout, device=dev)
    st = settings(args, 11)
    target = ds.forward(settings(args, 77), textures=[torch.as_tensor(tgt_tex, device=dev)]).clone()
    img = torch.empty_like(target)
    grad_img = torch.empty_like(target)
    g_tex = torch.zeros_like(ds.textures[0])
    g_rough = torch.zeros_like(ds.roughness)
    ck = Checkpoints(st.width * st.height * st.spp, st.max_depth)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # node / triangle visits of the forward's rays: the reverse sweep recomputes exactly these
    cf = torch.zeros(abi.PT_N_COUNTERS, dtype=torch.int64, device=dev)
    ds.forward(st, out=img, counters=cf)
    torch.cuda.synchronize()
    cf = cf.cpu().numpy()

    def prb(ev):
        ev[0].record(stream)
        ds.forward(st, out=img)
        torch.sub(img, target, out=grad_img)
        grad_img.mul_(2.0 / img.numel())
        ev[1].record(stream)
        ds.backward(st, grad_img, g_textures=[g_tex], g_roughness=g_rough, seed=12)
        ev[2].record(stream)

    def ckpt(ev):
        ev[0].record(stream)
        ckpt_forward(ds, st, ck, out=img)
        torch.sub(img, target, out=grad_img)
        grad_img.mul_(2.0 / img.numel())
        ev[1].record(stream)
        ckpt_backward(ds, st, ck, grad_img, g_textures=[g_tex], g_roughness=g_rough)
        ev[2].record(stream)

    dummy = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(max(3, args.warmup)):
        prb(dummy)
        ckpt(dummy)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    res = {"prb": [], "ckpt": []}
    for k in range(args.steps):
        for name, fn in (("prb", prb), ("ckpt", ckpt)):
            flush.fill_(float(k))
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            fn(ev)
            res[name].append(ev)
    torch.cuda.synchronize()
    clk = clocks.stop()

    def avg(name, a, b):
        return statistics.mean(e[a].elapsed_time(e[b]) for e in res[name])
    out = {k: {"forward_ms": round(avg(k, 0, 1), 3), "reverse_ms": round(avg(k, 1, 2), 3),
               "step_ms": round(avg(k, 0, 2), 3)} for k in res}
    line = {"metric": "gradient step: PRB vs reverse mode with checkpoints (ms, memory)",
            "value": round(out["ckpt"]["step_ms"] / out["prb"]["step_ms"], 3),
            "unit": "x time of the checkpointed step relative to the PRB step", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD["workload"] if not args.small else "spheres 256x256 64 spp",
                       "l2": "flushed before each timed step", "prb": out["prb"], "ckpt": out["ckpt"],
                       "ckpt_bytes": ck.nbytes, "prb_scratch_bytes": 0,
                       "prb_seed": "decorrelated (radiance pass + replay)",
                       "ckpt_seed": "the forward's (reverse sweep over stored vertices)"},
            "roofline": alu_roofline("ckpt_reverse_kernel", cf, args.bvh, out["ckpt"]["reverse_ms"], clk,
                                     "; the forward's rays, which the reverse sweep traces again"),
            "clocks": clk}
    print(json.dumps(line), flush=True)
    ck.close()


def run_reparam_experiment(args):
    """Reparameterized PRB (translation gradients of the 33 shapes through
    visibility) on the throughput scene at --reparam-spp samples per pixel: one
    gradient step = forward image, L2-loss image gradient, reparameterized
    adjoint (radiance pass + replay with the warps).  Rays = every ray the adjoint
    traces (radiance pass, replay, shadow, auxiliary and the warps' center rays,
    and the paths through pixel edges with their warps), counted by the kernels.
    Own JSON line."""
    import torch

    from paper_2202_01284_gb300 import abi
    from paper_2202_01284_gb300.render import DeviceScene
    from dataclasses import replace
    abi.load()
    dev = torch.device("cuda", 0)
    sc, tgt_tex = make_workload(small=args.small)
    layout = abi.PT_BVH_WIDE if args.bvh == "wide" else abi.PT_BVH_BINARY
    ds = DeviceScene(sc, layout=layout, device=dev)
    spp = 4 if args.small else args.reparam_spp
    st = replace(settings(args, 11), spp=spp, block_size=0, prb_mode=0)
    target = ds.forward(replace(st, seed=77), textures=[torch.as_tensor(tgt_tex, device=dev)]).clone()
    img = torch.empty_like(target)
    grad_img = torch.empty_like(target)
    g_t = torch.zeros((sc.n_shapes, 3), device=dev)
    rays = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev, count=None):
        ev[0].record(stream)
        ds.forward(st, out=img)
        torch.sub(img, target, out=grad_img)
        grad_img.mul_(2.0 / img.numel())
        ev[1].record(stream)
        ds.backward_reparam(replace(st, seed=12), grad_img, g_t, rays=count)
        ev[2].record(stream)

    dummy = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(max(3, args.warmup)):
        step(dummy)
    rays.zero_()
    step(dummy, rays)
    torch.cuda.synchronize()
    rays_step = int(rays.item())
    clocks = ClockSampler(0)
    clocks.start()
    evs = []
    for k in range(args.steps):
        flush.fill_(float(k))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        step(ev)
        evs.append(ev)
    torch.cuda.synchronize()
    clk = clocks.stop()
    fwd_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    rp_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    # node / triangle visits of the same launch (instrumented variant, after timing)
    cnt = torch.zeros(abi.PT_N_COUNTERS, dtype=torch.int64, device=dev)
    gt2 = torch.zeros_like(g_t)
    p = abi.params_struct(ds.albedo, ds.textures, ds.roughness, None)
    desc = ds._desc(ds.cameras, replace(st, seed=12), counters=cnt)
    abi.pt_render_backward_reparam(ds.handle, desc, p, abi.reparam_opts(), grad_img, gt2, None, stream.cuda_stream)
    # the radiance pass before the replay traces the forward's rays with the adjoint seed
    ds.forward(replace(st, seed=12), out=img, counters=cnt)
    torch.cuda.synchronize()
    c = cnt.cpu().numpy()
    flops = FLOPS_PER_NODE[args.bvh] * int(c[3]) + FLOPS_PER_TRI * int(c[4])
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 1477.0
    peak_tflops = sms * 128 * 2 * mhz * 1e6 / 1e12
    achieved = flops / (rp_ms / 1e3) / 1e12
    # the same estimator with every triangle corner's position as a parameter
    g_v = torch.zeros((sc.n_tris, 3, 3), device=dev)
    ev_v = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ds.backward_reparam(replace(st, seed=12), grad_img, g_vertices=g_v)
    flush.fill_(1.0)
    ev_v[0].record(stream)
    ds.backward_reparam(replace(st, seed=12), grad_img, g_vertices=g_v)
    ev_v[1].record(stream)
    torch.cuda.synchronize()
    vert_ms = ev_v[0].elapsed_time(ev_v[1])
    # forward mode along a direction over all shapes' translations (pt_render_jvp_reparam)
    direction = torch.ones((sc.n_shapes, 3), device=dev)
    jrays = torch.zeros(1, dtype=torch.int64, device=dev)
    ds.jvp_reparam(replace(st, seed=12), direction, with_image=False)
    flush.fill_(2.0)
    ev_j = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev_j[0].record(stream)
    ds.jvp_reparam(replace(st, seed=12), direction, with_image=False, rays=jrays)
    ev_j[1].record(stream)
    torch.cuda.synchronize()
    jvp_ms = ev_j[0].elapsed_time(ev_j[1])
    # the plain PRB adjoint of the same samples, for scale (texture + roughness gradients)
    g_tex = torch.zeros_like(ds.textures[0])
    g_rough = torch.zeros_like(ds.roughness)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ds.backward(replace(st, seed=12), grad_img, g_textures=[g_tex], g_roughness=g_rough)
    flush.fill_(0.0)
    e[0].record(stream)
    ds.backward(replace(st, seed=12), grad_img, g_textures=[g_tex], g_roughness=g_rough)
    e[1].record(stream)
    torch.cuda.synchronize()
    plain_ms = e[0].elapsed_time(e[1])
    opts = abi.reparam_opts()
    line = {"metric": "reparameterized PRB (shape-translation gradients through visibility), Mrays/s",
            "value": round(rays_step / rp_ms / 1e3, 2), "unit": "Mrays/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(fwd_ms + rp_ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": (f"spheres32x5120 + ground (196,608 tris, 33 shapes), {st.width}x{st.height}, "
                                    f"{spp} spp, depth 8, RR from 3; translation gradients of all 33 shapes"),
                       "l2": "flushed before each timed step", "forward_ms": round(fwd_ms, 3),
                       "reparam_adjoint_ms": round(rp_ms, 3), "plain_prb_adjoint_ms": round(plain_ms, 3),
                       "reparam_over_plain": round(rp_ms / plain_ms, 2), "rays_per_step": rays_step,
                       "vertex_mode_ms": round(vert_ms, 3),
                       "vertex_mode_mrays_s": round(rays_step / vert_ms / 1e3, 1),
                       "forward_mode_ms": round(jvp_ms, 3),
                       "forward_mode_mrays_s": round(int(jrays.item()) / jvp_ms / 1e3, 1),
                       "rays_per_sample": round(rays_step / (st.width * st.height * spp), 2),
                       "node_visits_per_ray": round(int(c[3]) / max(rays_step, 1), 2),
                       "tri_tests_per_ray": round(int(c[4]) / max(rays_step, 1), 2),
                       "options": {k: getattr(opts, k) for k, _ in opts._fields_},
                       "grad_translation_norm": float(g_t.norm().item())},
            "roofline": {"bound": "alu", "kernel": "reparam_kernel", "achieved": round(achieved, 3),
                         "peak": round(peak_tflops, 2), "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4),
                         "traffic": round(REPARAM_TRAFFIC_PER_SAMPLE * st.width * st.height * spp)
                                    if args.bvh == "wide" else None,
                         "traffic_basis": "ncu DRAM read + write per sample of reparam_kernel<1,0,0> at 256x256, "
                                          "4 spp (profiles/reparam_launches_spheres196k_256px_4spp.md), x samples",
                         "work": f"{FLOPS_PER_NODE[args.bvh]}/node visit + {FLOPS_PER_TRI}/triangle test (counted "
                                 "by instrumented launches of the replay, the pixel-edge paths and the radiance "
                                 "pass; warp-field arithmetic not counted); time = radiance pass + reparam_kernel "
                                 "+ edge_kernel",
                         "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x median SM clock {mhz} MHz"},
            "gpu_launches": (4 if opts.edge_spp > 0 else 3) * args.steps,  # forward, radiance pass, replay, edges
            "clocks": clk}
    print(json.dumps(line), flush=True)


MLP_FLOPS_PER_QUERY = 2 * (5 * 64 * 64 + 64 * 3)  # five 64x64 layers + the 64x3 head
# one training record: the forward, the head's and four hidden layers' input gradients
# (the encoding's is not needed) and all weight gradients
MLP_TRAIN_FLOPS_PER_RECORD = MLP_FLOPS_PER_QUERY + 2 * (64 * 3 + 4 * 64 * 64) + 2 * (5 * 64 * 64 + 64 * 3)


def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except Exception:
        return fallback, "fallback"


def run_mlp_experiment(args):
    """Radiance-cache MLP inference throughput: the tcgen05 engine (UMMA, TMEM
    accumulators) against the mma.sync engine on the same queries; then training
    throughput (Adam steps on 65,536-record batches) of both engines.  Own JSON line."""
    import numpy as np
    import torch

    from paper_2202_01284_gb300 import abi
    from paper_2202_01284_gb300 import scenes as S
    abi.load()
    n = (1 << 21) if args.small else (1 << 24)
    box = ((-1.0, 0.0, -1.0), (1.0, 2.0, 1.0))
    raw, _ = S.random_cache_records(min(n, 1 << 20), 3, *box)
    raw = np.tile(raw, (n // raw.shape[0], 1))
    h = abi.pt_cache_create(*box, batch=64, init_weights=S.mlp_init_weights(12))
    d_raw = torch.as_tensor(raw, device="cuda")
    d_out = torch.empty((n, 3), device="cuda")
    res = {}
    clocks = ClockSampler(0)
    clocks.start()
    for name, eng in (("tcgen05", abi.PT_CACHE_TCGEN05), ("mma_sync", abi.PT_CACHE_MMA_SYNC)):
        abi.pt_cache_set_engine(h, eng)
        for _ in range(max(3, args.warmup)):
            abi.pt_cache_query(h, d_raw, d_out, n)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            abi.pt_cache_query(h, d_raw, d_out, n)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        assert abi.pt_cache_status(h) == abi.PT_OK
        t = statistics.mean(ms)
        res[name] = {"ms": round(t, 4), "gqueries_s": round(n / t / 1e6, 3),
                     "tflops": round(n * MLP_FLOPS_PER_QUERY / t / 1e9, 1)}
    abi.pt_cache_destroy(h)
    # training: Adam steps on batches of 65,536 records (forward, backward deltas, weight
    # gradients, Adam), both engines, on the first 16 M records of the same set
    batch, tsteps = 65536, 16
    n_rec = batch * tsteps
    _, tgt = S.random_cache_records(min(n_rec, 1 << 20), 3, *box)
    tgt = np.tile(tgt, (n_rec // tgt.shape[0], 1))
    d_tgt = torch.as_tensor(tgt, device="cuda")
    train = {}
    for name, eng in (("tcgen05", abi.PT_CACHE_TCGEN05), ("mma_sync", abi.PT_CACHE_MMA_SYNC)):
        ht = abi.pt_cache_create(*box, batch=batch, init_weights=S.mlp_init_weights(12))
        abi.pt_cache_set_engine(ht, eng)
        for _ in range(max(3, args.warmup)):
            abi.pt_cache_train_records(ht, d_raw, d_tgt, n_rec, tsteps)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            abi.pt_cache_train_records(ht, d_raw, d_tgt, n_rec, tsteps)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        assert abi.pt_cache_status(ht) == abi.PT_OK
        abi.pt_cache_destroy(ht)
        t = statistics.mean(ms)
        train[name] = {"ms_per_adam_step": round(t / tsteps, 4), "mrecords_s": round(n_rec / t / 1e3, 1),
                       "tflops": round(n_rec * MLP_TRAIN_FLOPS_PER_RECORD / t / 1e9, 1)}
    clk = clocks.stop()
    peak, basis = measured_peak("bf16_tflops", 1900.0)
    ach = res["tcgen05"]["tflops"]
    line = {"metric": "radiance-cache MLP inference, queries/s (tcgen05 vs mma.sync)",
            "value": res["tcgen05"]["gqueries_s"], "unit": "G queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 (FP32 accumulate)", "data": "synthetic",
            "config": {"workload": f"{n} queries, 64-d encoding, 5x64 ReLU + 64x3, BF16 weights", "engines": res,
                       "speedup_over_mma_sync": round(res["mma_sync"]["ms"] / res["tcgen05"]["ms"], 2),
                       "training": {"batch": batch, "adam_steps": tsteps, "engines": train,
                                    "flops_per_record": MLP_TRAIN_FLOPS_PER_RECORD}},
            "roofline": {"bound": "tensor", "kernel": "nrc_infer_tc_kernel", "achieved": ach, "peak": peak,
                         "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": None,
                         "peak_basis": f"bf16 dense, {basis} (cuBLAS burst); includes the encoding on CUDA cores"},
            "clocks": clk}
    print(json.dumps(line), flush=True)


def cache_comparison(torch, warmup_frames=300, spps=(1, 2, 4, 8, 16, 32, 64, 96, 128, 192, 256, 320, 384),
                     bounces=(1, 2), plain_spp=64, ref_batches=16, ema=0.99):
    """Cornell box at 1024^2, depth 4: plain PT at `plain_spp` vs cache-terminated PT
    (bounce 1 and 2) at the spp that fits the same per-frame time including one online
    training update, after `warmup_frames` online training frames.  The network state
    (weights, Adam moments, step) after the warm-up is restored before every measured
    frame, so that every spp is judged with the same network (one identical online
    update inside each timed frame); without that, each measured frame trains on and
    the comparison drifts with the order of the sweep.  Reference: ref_batches x 256
    spp of plain PT with distinct seeds (the forward kernel, parity-tested against the
    FP64 oracle).  With ema > 0 the cache answers queries with the moving average of
    its weights (pt_cache_desc.ema), which is restored too."""
    from paper_2202_01284_gb300 import abi, scenes as S
    from paper_2202_01284_gb300.render import DeviceScene, RadianceCache, RenderSettings

    W, H, D = 1024, 1024, 4
    sc = S.cornell(width=W, height=H)
    ds = DeviceScene(sc, layout=abi.PT_BVH_WIDE)
    box = ((-1.0, 0.0, -1.0), (1.0, 2.0, 1.0))

    def st(spp, seed, **kw):
        return RenderSettings(width=W, height=H, spp=spp, max_depth=D, seed=seed, **kw)

    def timed(fn, reps=3, before=None):
        ts, out = [], None
        for _ in range(reps):
            if before:
                before()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record()
            out = fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts), out

    ref = torch.zeros((1, H, W, 3), device="cuda")
    for k in range(ref_batches):
        ref += ds.forward(st(256, 50000 + k))
    ref /= ref_batches
    # pixels that do not see the emitter (reference below 1): the light's edge pixels carry
    # anti-aliasing variance (radiance 15 vs ~0.2) that no cache can remove
    indirect = (ref.amax(dim=-1, keepdim=True) < 1.0).float()
    n_ind = float(indirect.sum()) * 3

    def mse(img):
        d2 = (img - ref) ** 2
        return float(d2.mean()), float((d2 * indirect).sum()) / n_ind

    t_plain, img_plain = timed(lambda: ds.forward(st(plain_spp, 7)))
    mp, mpi = mse(img_plain)
    out = {"metric": "equal-time MSE vs the reference, radiance cache vs plain PT",
           "workload": f"cornell36, {W}x{H}, depth {D}", "reference_spp": 256 * ref_batches,
           "indirect_pixel_fraction": round(n_ind / (3 * W * H), 4),
           "plain": {"spp": plain_spp, "ms": round(t_plain, 3), "mse": mp, "mse_indirect": mpi}}
    for bounce in bounces:
        cache = RadianceCache(*box, batch=65536, max_queries=W * H * max(spps), max_records=2_000_000,
                              max_paths=256 * 256, lr=5e-3, init_weights=S.mlp_init_weights(2022), ema=ema)
        train_st = RenderSettings(width=256, height=256, spp=1, max_depth=D, seed=0)
        train_cam = [S.cornell_camera(256, 256)]

        def train_frame(i):
            train_st.seed = 900000 + i
            return cache.train(ds, train_st, steps=4, cams=train_cam)
        t0 = time.perf_counter()
        for i in range(warmup_frames):
            train_frame(i)
        torch.cuda.synchronize()
        warm_s = time.perf_counter() - t0
        loss = cache.last_loss()
        state = abi.pt_cache_get_state(cache.handle)
        avg = cache.average()

        def restore():
            abi.pt_cache_set_state(cache.handle, *state)
            cache.set_average(avg)
        res, best = {}, None
        for spp in spps:
            t_frame, img = timed(lambda: (train_frame(10 ** 6),
                                          ds.forward(st(spp, 8, cache=cache.handle, cache_bounce=bounce)))[1],
                                 before=restore)
            m_all, m_ind = mse(img)
            res[spp] = {"ms": round(t_frame, 3), "mse": m_all, "mse_indirect": m_ind}
            if t_frame <= t_plain:
                best = spp
        eq = res[best] if best else None
        out[f"cache_bounce{bounce}"] = {
            "warmup_frames": warmup_frames, "warmup_s": round(warm_s, 2), "train_loss": loss,
            "per_frame": "one pt_cache_train (256^2 training paths, 1 spp, 4 Adam steps of 65,536) + render; "
                         "network state restored before each measured frame",
            "weight_average": ema,
            "equal_time_spp": best, "equal_time": eq,
            "mse_indirect_ratio_plain_over_cache": (mpi / eq["mse_indirect"]) if eq else None,
            "mse_ratio_plain_over_cache": (mp / eq["mse"]) if eq else None,
            "sweep": res}
        cache.close()
    return out


def run_cache_experiment(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(cache_comparison(torch, warmup_frames=args.cache_warmup_frames, ema=args.cache_ema)), flush=True)


def run_batch_experiment(args):
    """64 cameras (128^2..1024^2, 4..64 spp) over three sphere scenes of ~10k, ~200k and
    ~2M triangles: forward + PRB adjoint (L2 loss vs a constant 0.3 target, gradients into
    each scene's texture and roughness) as one persistent launch replayed from a CUDA
    graph with autotuned tiles, vs 64 x (forward, loss gradient, backward) launches."""
    import torch

    from paper_2202_01284_gb300 import abi, batch as B, scenes as S
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    scenes = [DeviceScene(sc, layout=abi.PT_BVH_WIDE) for sc in S.batch_scenes()]
    setup_s = time.perf_counter() - t0
    cams = S.batch_cameras(64)
    g_tex = [[torch.zeros_like(t) for t in ds.textures] for ds in scenes]
    g_rough = [torch.zeros_like(ds.roughness) for ds in scenes]

    def reset():
        for gl in g_tex:
            for g in gl:
                g.zero_()
        for g in g_rough:
            g.zero_()
    jobs = []
    for k, bc in enumerate(cams):
        tgt = torch.full((bc.camera.height, bc.camera.width, 3), 0.3, device="cuda")
        jobs.append(B.Job(scenes[bc.scene], bc.camera, bc.spp, seed=10 + k, backward_seed=5000 + k, target=tgt,
                          g_textures=g_tex[bc.scene], g_roughness=g_rough[bc.scene]))
    samples = sum(j.camera.width * j.camera.height * j.spp for j in jobs)
    grad_bufs = {(j.camera.height, j.camera.width): torch.empty((j.camera.height, j.camera.width, 3), device="cuda")
                 for j in jobs}
    # rays of the whole workload (instrumented separate launches of the same jobs)
    cnt_f = torch.zeros(abi.PT_N_COUNTERS, dtype=torch.int64, device="cuda")
    cnt_b = torch.zeros(abi.PT_N_COUNTERS, dtype=torch.int64, device="cuda")

    def st_of(j):
        return RenderSettings(width=j.camera.width, height=j.camera.height, spp=j.spp, max_depth=j.max_depth,
                              rr_depth=j.rr_depth, seed=j.seed, lanes_per_pixel=min(8, j.spp))

    def separate(counters=False):
        for j in jobs:
            st = st_of(j)
            img = j.dscene.forward(st, cams=[j.camera], out=j.image[None], counters=cnt_f if counters else None)
            torch.sub(img[0], j.target, out=grad_bufs[j.camera.height, j.camera.width])
            gi = grad_bufs[j.camera.height, j.camera.width]
            gi.mul_(2.0 / img.numel())
            j.dscene.backward(st, gi[None], cams=[j.camera], g_textures=j.g_textures,
                              g_roughness=j.g_roughness, seed=j.backward_seed, counters=cnt_b if counters else None)
    separate(counters=True)
    torch.cuda.synchronize()
    rays = int(cnt_f[1] + cnt_f[2] + cnt_b[1] + cnt_b[2])
    reset()

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, e = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(e))
        return statistics.median(ts)
    sep_ms = timed(separate)
    reset()
    best = B.autotune(jobs, candidates=[(t, l, c) for t in (2, 4, 8) for l in (2, 4, 8) for c in (4, 8)],
                      use_cache=False, reset_grads=reset)
    b = B.Batch(jobs, tile=best["tile"], lanes_per_pixel=best["lanes_per_pixel"], ctas_per_sm=best["ctas_per_sm"])
    b.capture()
    clocks = ClockSampler(0)
    clocks.start()
    graph_ms = timed(b.replay)
    clk = clocks.stop()
    direct_ms = timed(b.run)
    out = {"metric": "batched forward + adjoint: one persistent CUDA-graph launch vs 64 separate launches",
           "jobs": len(jobs), "scenes_tris": [ds.scene.n_tris for ds in scenes], "samples": samples, "rays": rays,
           "work_items": b.n_items, "scene_setup_s": round(setup_s, 2),
           "persistent_graph_ms": round(graph_ms, 3), "persistent_direct_ms": round(direct_ms, 3),
           "separate_ms": round(sep_ms, 3), "speedup": round(sep_ms / graph_ms, 3),
           "mrays_s_persistent": round(rays / graph_ms / 1e3, 1), "mrays_s_separate": round(rays / sep_ms / 1e3, 1),
           "gpu_launches": {"persistent": 3, "separate": 3 * len(jobs), "graph_launches": 1},
           "autotune": {k: v for k, v in best.items() if k != "candidates"},
           "autotune_candidates": best["candidates"]}
    cnt = (cnt_f + cnt_b).cpu().numpy()
    out["roofline"] = alu_roofline("batch_kernel (forward, radiance pass, replay)", cnt, "wide", graph_ms, clk,
                                   "; every job's forward and adjoint rays over the graph's time")
    out["clocks"] = clk
    print(json.dumps(out), flush=True)


def measure_roofs(torch, dev=0, l2_mb=48, reps=20):
    """Memory-side roofs with the library's own probes (pt_probe_read / pt_probe_atomic),
    timed with CUDA events on the stream they run on: L2-resident and HBM-sized 16-byte
    reads, and fire-and-forget float / float4 atomic adds spread over the texture-gradient
    buffer size (1M float4) or colliding on 96 floats (the roughness gradients)."""
    from paper_2202_01284_gb300 import abi
    stream = torch.cuda.current_stream(dev)

    def t_ms(fn, n=reps):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / n
    sink = torch.zeros(1, device=dev)
    out = {}
    buf = torch.rand(l2_mb * (1 << 20) // 4, device=dev)
    ms = t_ms(lambda: abi.pt_probe_read(buf, 4, sink, stream.cuda_stream))
    out["l2_read_gbs"] = round(buf.numel() * 4 * 4 / ms / 1e6, 1)
    del buf
    big = torch.empty((4 << 30) // 4, device=dev)
    big.fill_(1.0)
    ms = t_ms(lambda: abi.pt_probe_read(big, 1, sink, stream.cuda_stream), n=5)
    out["hbm_read_gbs"] = round(big.numel() * 4 / ms / 1e6, 1)
    del big
    n = 1 << 24
    dst = torch.zeros((1 << 20) * 4, device=dev)
    ms = t_ms(lambda: abi.pt_probe_atomic(dst, 1 << 20, n, 4, stream.cuda_stream), n=5)
    out["red_f4_spread_1M_gops"] = round(n / ms / 1e6, 2)
    ms = t_ms(lambda: abi.pt_probe_atomic(dst, 1 << 20, n, 1, stream.cuda_stream), n=5)
    out["red_f1_spread_1M_gops"] = round(n / ms / 1e6, 2)
    ms = t_ms(lambda: abi.pt_probe_atomic(dst, 96, n, 1, stream.cuda_stream), n=3)
    out["red_f1_colliding_96_gops"] = round(n / ms / 1e6, 2)
    out["basis"] = (f"pt_probe_read: {l2_mb} MB x 4 passes (L2-resident), 4 GB x 1 pass (HBM), 16-B L2-only loads; "
                    "pt_probe_atomic: 16M adds; CUDA events, mean of repeated launches")
    return out


def run_peaks(args):
    """Memory-side roofs measured with the library's own probes."""
    import torch
    torch.cuda.set_device(0)
    out = {"metric": "memory-side roofs (own microbenchmarks)", **measure_roofs(torch)}
    props = torch.cuda.get_device_properties(0)
    out["sms"] = props.multi_processor_count
    out["fp32_peak_tflops_at_2070mhz"] = round(props.multi_processor_count * 128 * 2 * 2070e6 / 1e12, 2)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.peaks:
        run_peaks(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.cache:
        run_cache_experiment(args)
    elif args.batch:
        run_batch_experiment(args)
    elif args.jvp:
        run_jvp_experiment(args)
    elif args.wavefront:
        run_wavefront_experiment(args)
    elif args.ckpt:
        run_ckpt_experiment(args)
    elif args.reparam:
        run_reparam_experiment(args)
    elif args.trace:
        run_trace_experiment(args)
    elif args.texgrad:
        run_texgrad_experiment(args)
    elif args.mlp:
        run_mlp_experiment(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
