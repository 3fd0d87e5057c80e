#!/usr/bin/env python
"""Benchmark of the GB300 2D Gaussian ray tracer (one JSON line on rank 0).

Workload (one GPU): the camera-ray scene-scale configuration -- 300k surfels
on a synthetic object scene (unit sphere, torus, ground square; tangent with
1% normal jitter; log-normal scales with median 0.01; opacity Beta(5,1);
10 feature channels) traced by 100 cameras x 800x800 = 64M rays, k = 16.
A step is the training-style pass over that batch: rebuild the scene's LBVH
from the surfel values (K1-K5), trace all rays forward (Eq. 8) and run the
backward pass for a random N(0,1) upstream gradient. `value` is rays traced
forward and backward per second (Mrays/s), inputs resident on the device.
The Monte Carlo rendering-equation configuration (1M surfels, 640k points x
64 samples = 41M secondary rays) is timed in the same run under "mc".

`--impl reference` times the FP64 CPU oracle (there is no reference implementation to run)
on bounded samples of the same workload, on the host cores.

Run with torchrun for N > 1: each rank traces its own 100-camera batch
(weak scaling) and the surfel gradients are summed across ranks (the one
exchange step of a data-parallel backward).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s traced+composited (fwd, fwd+bwd) vs roofline; served p50/p99 latency"
UNIT = "Mrays/s"
WORKLOAD = "camera rays at scene scale: 300k-surfel object scene, 100 cameras x 800x800, k=16, 10 channels"

# FP32 pipe of one GB300: 152 SMs x 128 FP32 lanes x 2 flops (FMA) at the
# 2070 MHz maximum SM clock.
SMS, LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SMS * LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12

# DRAM traffic per launch of the dominant kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) scaled per ray; keyed by
# the hash of the sources it was measured on, the hierarchy's builder
# included (null once they change).
# Captured on the 10-camera case (6.4M rays; the ~90 MB scene read is ~5% of
# it, so the per-ray figure slightly overstates a 64M-ray launch).
TRAFFIC = {
    # the four round launches of one forward (6.4M-ray capture): read 428.9 + 919.9 + 358.2 + 87.1 MB,
    # written 756.3 + 561.3 + 125.0 + 11.7 MB
    "k_trace_round<16,10,*>": {"bytes_per_ray": (1794.1e6 + 1454.3e6) / 6.4e6, "src_hash": "99bbb098cc97"},
}


def _kernel_hash(files):
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2412_15867_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cams", type=int, default=100)
    ap.add_argument("--res", type=int, default=800)
    ap.add_argument("--surfels", type=int, default=300_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--saved-hits", type=int, default=96,
                    help="hit-list length the forward saves for the backward (0: the backward replays)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mc", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-raster", action="store_true")
    ap.add_argument("--serve-only", action="store_true", help="run only the serving leg")
    ap.add_argument("--mc-only", action="store_true", help="run only the Monte Carlo shading leg")
    ap.add_argument("--mc-points", type=int, default=640_000)
    ap.add_argument("--mc-surfels", type=int, default=1_000_000)
    ap.add_argument("--mc-reps", type=int, default=2)
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--serve-warmup", type=float, default=2.0)
    ap.add_argument("--cpu-rays", type=int, default=20480, help="oracle sample for cpu_baseline")
    ap.add_argument("--ref-rays", type=int, default=1024, help="oracle rays per reference step")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": sorted(reasons)}


def algorithmic_flops(nh, k, n_surfels, F, backward=False, saved_hits=0):
    """Algorithmic FP32 flops of one launch: per composited hit one Eq. 6-7
    intersection (45, exp counted as 1) plus blending (2(F+2) + 3); per
    k-buffer round one root-to-leaf descent of ceil(log2 N) nodes with two
    slab tests (40). The backward costs about 3x per hit and descends only
    for rays whose hit list was not saved (n_hits > saved_hits)."""
    import torch
    nh = nh.to(torch.float64)
    rounds = torch.floor(nh / k) + 1
    per_hit = 45 + 2 * (F + 2) + 3
    depth = math.ceil(math.log2(max(n_surfels, 2)))
    if backward and saved_hits > 0:
        rounds = torch.where(nh > saved_hits, rounds, torch.zeros_like(rounds))
    f = nh * per_hit * (3 if backward else 1) + rounds * depth * 40
    return float(f.sum())


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_2412_15867_gb300 as irgs
    from paper_2412_15867_gb300 import _lib
    from paper_2412_15867_gb300.dist import allreduce_grads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = _lib.lib()

    # ---- synthetic workload (same scene on every rank, own cameras per rank)
    sc = synth.object_scene(args.surfels, seed=1001)
    cams = synth.hemisphere_cameras(args.cams, seed=1001 + 7919 * rank)
    # pixels in 4x8 tiles (4 wide, 8 tall): a warp's 32 rays cover a compact patch of the image
    ro_np, rd_np = synth.camera_batch_rays(cams, args.res, args.res, tile=(4, 8))
    R = ro_np.shape[0]
    F = sc.features.shape[1]
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    surf = [T(a) for a in sc.arrays()]
    ro, rd = T(ro_np), T(rd_np)
    gf_np, gd_np, go_np = synth.upstream_grads(R, F, seed=1004 + rank)
    gf, gd, go = T(gf_np), T(gd_np), T(go_np)
    p = irgs.TraceParams(k=16, feat_count=F)
    scene = irgs.Scene(*surf, alpha_min=1 / 255)
    # the forward keeps each ray's hit list (4 B per blended hit) so that the
    # backward needs no second traversal; rays with more hits replay it
    out = irgs.trace_forward(scene, ro, rd, p, max_hit_ids=args.saved_hits)
    grads = {"means": torch.zeros((sc.n, 3), device=dev), "quats": torch.zeros((sc.n, 4), device=dev),
             "scales": torch.zeros((sc.n, 2), device=dev), "opacity": torch.zeros(sc.n, device=dev),
             "features": torch.zeros((sc.n, F), device=dev)}
    stream = torch.cuda.current_stream(dev)

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        scene.update()
        if evs:
            evs[1].record(stream)
        irgs.trace_forward(scene, ro, rd, p, max_hit_ids=args.saved_hits, out=out)
        if evs:
            evs[2].record(stream)
        for g in grads.values():
            g.zero_()
        irgs.trace_backward(scene, ro, rd, p, out, gf, gd, go, grads=grads)
        if evs:
            evs[3].record(stream)
        if world > 1:
            allreduce_grads(grads)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if scene.status() != 0:
        raise RuntimeError("device error during warm-up")

    clocks = ClockSampler(local)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = L.irgs_kernel_launches()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    launches = L.irgs_kernel_launches() - launches0
    total_ms = t_start.elapsed_time(t_end)
    build_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    fwd_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    bwd_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    tmax = torch.tensor([total_ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    total_ms = float(tmax.item())
    ms_per_step = total_ms / args.steps
    value = R * world * args.steps / (total_ms * 1e-3) / 1e6
    if scene.status() != 0:
        raise RuntimeError("device error in the timed region")

    # ---- refit-only BVH update (same surfels: keeps the rebuilt tree's quality)
    ra, rb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ra.record(stream)
    for _ in range(5):
        scene.refit()
    rb.record(stream)
    torch.cuda.synchronize()
    refit_ms = ra.elapsed_time(rb) / 5

    # ---- the radix-tree hierarchy on the same surfels and rays, for comparison
    # (rebuild and forward, two runs each after one warm-up; the timed step
    # above uses the clustered hierarchy)
    hier = None
    if rank == 0:
        rscene = irgs.Scene(*surf, alpha_min=1 / 255, hierarchy="radix")
        irgs.trace_forward(rscene, ro, rd, p, max_hit_ids=args.saved_hits, out=out)
        hb = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        hb[0].record(stream)
        for _ in range(2):
            rscene.update()
        hb[1].record(stream)
        for _ in range(2):
            irgs.trace_forward(rscene, ro, rd, p, max_hit_ids=args.saved_hits, out=out)
        hb[2].record(stream)
        torch.cuda.synchronize()
        if rscene.status() != 0:
            raise RuntimeError("device error on the radix-tree scene")
        hier = {"clustered": {"build_ms": build_ms, "fwd_ms": fwd_ms},
                "radix": {"build_ms": hb[0].elapsed_time(hb[1]) / 2, "fwd_ms": hb[1].elapsed_time(hb[2]) / 2}}
        rscene.close()

    # ---- 2D Gaussian rasterisation of the same cameras (the G-buffer pass of stage II)
    raster = None
    if not args.no_raster and rank == 0:
        from paper_2412_15867_gb300 import serve as _serve
        n_cam = min(args.cams, 20)
        rcams = [_serve.make_camera(e, args.res, args.res, fov_deg=60.0) for e in cams[:n_cam]]
        pr = irgs.TraceParams(k=16, feat_count=F)
        ro_ = irgs.rasterize(scene, rcams[0], pr)
        torch.cuda.synchronize()
        ra.record(stream)
        for c_ in rcams:
            irgs.rasterize(scene, c_, pr, out=ro_)
        rb.record(stream)
        torch.cuda.synchronize()
        r_ms = ra.elapsed_time(rb) / n_cam
        raster = {"workload": f"{n_cam} of the cameras, {args.res}x{args.res}, {F} channels, 16x16 tiles",
                  "ms_per_image": r_ms, "mpix_s": args.res * args.res / (r_ms * 1e-3) / 1e6,
                  "traced_ms_per_image": fwd_ms / args.cams}

    # ---- roofline of the dominant kernel (by time)
    nh = out["n_hits"]
    if bwd_ms >= fwd_ms:
        kname, kms = "k_trace_backward<16,10>", bwd_ms
        flops = algorithmic_flops(nh, 16, sc.n, F, backward=True, saved_hits=args.saved_hits)
        src = ["trace.cuh", "trace_bwd.cuh", "trace_bwd.cu", "common.cuh", "scene.cu"]
    else:
        # the forward pass: for batches of 2^20 rays or more its compacted
        # k-buffer rounds (4 launches) and the compaction between them
        kname, kms = "k_trace_round<16,10,*>", fwd_ms
        flops = algorithmic_flops(nh, 16, sc.n, F)
        src = ["trace.cuh", "trace_fwd.cu", "common.cuh", "scene.cu"]
    achieved = flops / (kms * 1e-3) / 1e12
    khash = _kernel_hash(src)
    tr = TRAFFIC.get(kname)
    traffic = tr["bytes_per_ray"] * R if (tr and tr.get("bytes_per_ray") and tr.get("src_hash") == khash) else None
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                "flops_per_launch": flops, "launch_ms": kms,
                "peak_note": "152 SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz max SM clock",
                "hbm_bound_mrays_s": None}

    # ---- end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        host_in = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                   for k, a in zip(("means", "quats", "scales", "opacity", "features"), sc.arrays())}
        host_in.update({"ro": torch.from_numpy(ro_np).pin_memory(), "rd": torch.from_numpy(rd_np).pin_memory(),
                        "gf": torch.from_numpy(gf_np).pin_memory(), "gd": torch.from_numpy(gd_np).pin_memory(),
                        "go": torch.from_numpy(go_np).pin_memory()})
        dev_in = {k: torch.empty_like(v, device=dev) for k, v in host_in.items()}
        # the rendered outputs and the gradients come back; the hit lists stay on the device
        host_out = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in out.items() if k != "hit_ids"}
        host_out.update({("g_" + k): torch.empty_like(v, device="cpu").pin_memory() for k, v in grads.items()})
        h2d = sum(v.numel() * v.element_size() for v in host_in.values())
        d2h = sum(v.numel() * v.element_size() for v in host_out.values())
        scene_e2e = irgs.Scene(dev_in["means"], dev_in["quats"], dev_in["scales"], dev_in["opacity"],
                               dev_in["features"])

        # pipelined by camera chunks: host->device copies of chunk c+1 and
        # device->host copies of chunk c-1 overlap the traces of chunk c
        n_chunk = max(1, min(10, args.cams))
        bounds_ = [(R * i // n_chunk, R * (i + 1) // n_chunk) for i in range(n_chunk)]
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(n_chunk)]
        ev_done = [torch.cuda.Event() for _ in range(n_chunk)]
        ev_out = torch.cuda.Event()
        scene_keys = ("means", "quats", "scales", "opacity", "features")
        ray_keys = ("ro", "rd", "gf", "gd", "go")

        def e2e_step():
            s_in.wait_stream(stream)
            s_out.wait_stream(stream)
            for k in scene_keys:
                dev_in[k].copy_(host_in[k], non_blocking=True)
            with torch.cuda.stream(s_in):
                for i, (lo, hi) in enumerate(bounds_):
                    for k in ray_keys:
                        dev_in[k][lo:hi].copy_(host_in[k][lo:hi], non_blocking=True)
                    ev_in[i].record(s_in)
            scene_e2e.update()
            for g in grads.values():
                g.zero_()
            for i, (lo, hi) in enumerate(bounds_):
                stream.wait_event(ev_in[i])
                sl = {k: out[k][lo:hi] for k in out}
                irgs.trace_forward(scene_e2e, dev_in["ro"][lo:hi], dev_in["rd"][lo:hi], p,
                                   max_hit_ids=args.saved_hits, out=sl)
                irgs.trace_backward(scene_e2e, dev_in["ro"][lo:hi], dev_in["rd"][lo:hi], p, sl,
                                    dev_in["gf"][lo:hi], dev_in["gd"][lo:hi], dev_in["go"][lo:hi], grads=grads)
                ev_done[i].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done[i])
                    for k in ("feat", "depth", "opacity", "n_hits"):
                        host_out[k][lo:hi].copy_(out[k][lo:hi], non_blocking=True)
            for k, v in grads.items():
                host_out["g_" + k].copy_(v, non_blocking=True)
            ev_out.record(s_out)
            stream.wait_event(ev_out)

        e2e_step()
        torch.cuda.synchronize()
        n_e2e = max(2, args.steps)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n_e2e):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = a.elapsed_time(b) / n_e2e
        e2e = {"value": R * world / (e_ms * 1e-3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e_ms,
               "pipeline": f"{n_chunk} camera chunks; copies on two side streams overlap the traces"}
        scene_e2e.close()

    # ---- Monte Carlo rendering equation configuration
    mc = None
    if not args.no_mc and rank == 0:
        mc = mc_leg(args, dev)

    # ---- serving mix (continuous batching vs one request at a time)
    serving = None
    if not args.no_serve and rank == 0:
        del out, grads, ro, rd, gf, gd, go
        torch.cuda.empty_cache()
        serving = serve_leg(args, dev)

    # ---- oracle on the host cores, bounded sample of the same workload
    cpu = None
    if not args.no_cpu and rank == 0:
        cpu = cpu_baseline(sc, ro_np, rd_np, gf_np, gd_np, go_np, args.cpu_rays)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded object scene and camera rays; no dataset)",
            "config": {"workload": WORKLOAD, "surfels": sc.n, "rays_per_step_per_gpu": R,
                       "cameras": args.cams, "resolution": args.res, "k": 16, "feat_count": F,
                       "alpha_min": 1 / 255, "T_min": 1e-4,
                       "step": "BVH rebuild (Morton sort, clustered binary tree, 4-wide collapse) + forward trace (saving hit lists) + backward trace from the lists",
                       "saved_hits": args.saved_hits,
                       "ray_order": "4x8 pixel tiles per camera (4 wide, 8 tall; one warp each)", "traversal": "warp-coherent",
                       "l2": "inputs larger than L2 (1.5 GB of rays per step)"},
            "fwd_mrays_s": R / (fwd_ms * 1e-3) / 1e6, "bwd_mrays_s": R / (bwd_ms * 1e-3) / 1e6,
            "build_ms": build_ms, "refit_ms": refit_ms, "fwd_ms": fwd_ms, "bwd_ms": bwd_ms, "hierarchies": hier,
            "mean_hits_per_ray": float(nh.float().mean()), "max_hits_per_ray": int(nh.max()),
            "replayed_ray_frac": float((nh > args.saved_hits).float().mean()) if args.saved_hits > 0 else 1.0,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk, "raster": raster, "mc": mc, "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def mc_leg(args, dev):
    """Monte Carlo rendering equation at G-buffer points (Eq. 13-15): object
    scene of --mc-surfels surfels (1M), --mc-points points (640k) x (32
    cosine + 32 GGX) secondary rays, 512x256 environment, k=16. Times the
    shading forward and its gradient (surfels, albedo, roughness, env)."""
    import numpy as np
    import torch
    import synth
    import paper_2412_15867_gb300 as irgs

    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.current_stream(dev)
    Pn = args.mc_points
    sc2 = synth.object_scene(args.mc_surfels, seed=1002)
    gb = synth.gbuffer_points(Pn, seed=1002)
    env = T(synth.env_map(seed=1003))
    S2 = irgs.Scene(*(T(a) for a in sc2.arrays()))
    g2 = [T(a) for a in gb]
    ps = irgs.TraceParams(k=16, feat_count=3, t_min=1e-3)
    g_rgb = T(np.random.default_rng(1004).normal(size=(Pn, 3)).astype(np.float32))
    o2 = irgs.shade_mc(S2, *g2, env, 32, 32, 2024, ps)
    gr = irgs.shade_mc_backward(S2, *g2, env, 32, 32, 2024, ps, g_rgb)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    reps = args.mc_reps
    ev[0].record(stream)
    for _ in range(reps):
        irgs.shade_mc(S2, *g2, env, 32, 32, 2024, ps, out=o2)
    ev[1].record(stream)
    for _ in range(reps):
        for g in gr.values():
            g.zero_()
        irgs.shade_mc_backward(S2, *g2, env, 32, 32, 2024, ps, g_rgb, grads=gr)
    ev[2].record(stream)
    torch.cuda.synchronize()
    fms = ev[0].elapsed_time(ev[1]) / reps
    bms = ev[1].elapsed_time(ev[2]) / reps
    # the fused kernel (a warp per point tracing its own samples), for reference
    pf = ps.with_(flags=irgs.FLAG_PER_THREAD)
    ev[0].record(stream)
    irgs.shade_mc(S2, *g2, env, 32, 32, 2024, pf, out=o2)
    ev[1].record(stream)
    torch.cuda.synchronize()
    fused_ms = ev[0].elapsed_time(ev[1])
    rays = Pn * 64
    # relighting query under a new environment: pre-integration, then
    # 64 environment-importance samples per point tracing albedo/roughness/normal
    env_new = T(synth.env_map(seed=1005))
    ev[0].record(stream)
    E = irgs.EnvMap(env_new)
    ev[1].record(stream)
    pr = irgs.TraceParams(k=16, feat_offset=3, feat_count=7, t_min=1e-3)
    orl = irgs.relight(S2, E, *g2, 64, 2025, pr)
    ev[2].record(stream)
    torch.cuda.synchronize()
    env_ms = ev[0].elapsed_time(ev[1])
    ev[0].record(stream)
    for _ in range(reps):
        irgs.relight(S2, E, *g2, 64, 2025, pr, out=orl)
    ev[1].record(stream)
    torch.cuda.synchronize()
    relight_ms = ev[0].elapsed_time(ev[1]) / reps
    E.close()
    if S2.status() != 0:
        raise RuntimeError("device error in the MC leg")
    S2.close()
    return {"workload": f"{args.mc_surfels} surfels, {Pn} G-buffer points x (32 cosine + 32 GGX) = "
                        f"{rays / 1e6:.1f}M secondary rays, 512x256 env, k=16",
            "ms": fms, "mrays_s": rays / (fms * 1e-3) / 1e6, "points_per_s": Pn / (fms * 1e-3),
            "bwd_ms": bms, "bwd_mrays_s": rays / (bms * 1e-3) / 1e6,
            "path": "secondary rays regrouped by direction bin and origin Morton code, one stack per ray",
            "fused_per_lane_ms": fused_ms,
            "relight": {"workload": f"{Pn} points x 64 environment-importance samples, 512x256 environment, "
                                    "traced albedo/roughness/normal shaded with split-sum maps",
                        "envmap_ms": env_ms, "ms": relight_ms, "mrays_s": rays / (relight_ms * 1e-3) / 1e6}}


def serve_leg(args, dev):
    """Serving mix: 4 resident scenes (100k, 300k, 1M, 2M surfels, object scene
    with median scale 0.01 sqrt(300k/N)); 50% render (camera rays, 10
    channels) / 50% relight (G-buffer + Monte Carlo shading, spp log-uniform
    in [1, 128]) requests at resolutions {128, 256, 512, 1024}^2 from random
    hemisphere cameras. Saturated throughput first (all requests queued at
    once), then a Poisson stream at 0.7x that rate served with continuous
    batching and, separately, one request at a time."""
    import numpy as np
    import torch
    import synth
    import paper_2412_15867_gb300 as irgs
    from paper_2412_15867_gb300 import serve

    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sizes = [100_000, 300_000, 1_000_000, 2_000_000]
    scenes = [irgs.Scene(*(T(a) for a in synth.object_scene(n, seed=1010 + i).arrays())) for i, n in enumerate(sizes)]
    env = T(synth.env_map(seed=1003))
    res = [128, 256, 512, 1024]

    def maker(seed):
        rng = np.random.default_rng(seed)

        def make(i):
            scene = int(rng.integers(0, 4))
            r = res[int(rng.integers(0, 4))]
            z = rng.uniform(np.sin(np.radians(5)), 1.0)
            ph = rng.uniform(0, 2 * np.pi)
            eye = (4 * np.sqrt(1 - z * z) * np.cos(ph), 4 * np.sqrt(1 - z * z) * np.sin(ph), 4 * z)
            if rng.uniform() < 0.5:
                return serve.RenderRequest(scene, eye, r, r)
            spp = int(np.clip(np.round(np.exp(rng.uniform(0, np.log(128)))), 1, 128))
            return serve.RelightRequest(scene, eye, r, r, spp=spp, env=env, seed=int(rng.integers(1 << 62)))
        return make

    budget = 24 << 30
    # saturated: a burst of requests served with continuous batching
    srv = serve.Server(scenes, hbm_budget=budget, max_jobs=64, max_tiles=8192)
    mk = maker(11)
    n_burst = 48
    for i in range(4):                                   # warm-up (graph capture, caches)
        srv.submit(mk(i))
    srv.run_until_idle()
    rays0 = srv.rays_total
    t0 = time.perf_counter()
    burst = [srv.submit(mk(100 + i), arrival=t0) for i in range(n_burst)]
    srv.run_until_idle()
    sat_wall = time.perf_counter() - t0
    sat_rate = n_burst / sat_wall
    sat_mrays = (srv.rays_total - rays0) / sat_wall / 1e6
    rate = 0.7 * sat_rate
    out = {"scenes_surfels": sizes, "mix": "50% render (10 ch) / 50% relight (spp log-uniform 1-128), "
           "res {128,256,512,1024}^2, random hemisphere cameras, Poisson arrivals",
           "saturated": {"requests_per_s": sat_rate, "mrays_s": sat_mrays, "requests": n_burst},
           "rate_requests_per_s": rate}
    for name, batching in (("batched", True), ("one_at_a_time", False)):
        srv2 = serve.Server(scenes, hbm_budget=budget, max_jobs=64, max_tiles=8192, batching=batching)
        hs, wall, rays = serve.run_poisson(srv2, maker(23), rate, args.serve_seconds, args.serve_warmup, seed=5)
        st = serve.latency_stats(hs)
        st.update({"mrays_s": rays / wall / 1e6, "requests_per_s": len(hs) / wall, "steps": srv2.steps})
        out[name] = st
        srv2.close()
    status = sum(S.status() for S in scenes)
    if status:
        raise RuntimeError("device error in the serving leg")
    srv.close()
    for S in scenes:
        S.close()
    return out


def cpu_baseline(sc, ro, rd, gf, gd, go, n_rays):
    """Oracle forward + gradient on a seeded sample of the workload's rays."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(99)
    idx = np.sort(rng.choice(ro.shape[0], n_rays, replace=False))
    p = oracle.Params(feat_count=sc.features.shape[1])
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    oracle.trace(sc, ro[idx], rd[idx], p, margins=None)
    oracle.trace_grad(sc, ro[idx], rd[idx], gf[idx], gd[idx], go[idx], p)
    dt = time.perf_counter() - t0
    return {"value": n_rays / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_rays} seeded camera rays of the workload, forward + gradient, FP64 brute force "
                      f"over all {sc.n} surfels ({dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    import synth
    sc = synth.object_scene(args.surfels, seed=1001)
    cams = synth.hemisphere_cameras(args.cams, seed=1001)
    rng = np.random.default_rng(5)
    p = oracle.Params(feat_count=sc.features.shape[1])
    cores = oracle.num_threads()
    ci = rng.integers(0, args.cams, size=args.ref_rays)
    # rays of random pixels of random cameras of the workload
    ro_l, rd_l = [], []
    for c in np.unique(ci):
        o, d = synth.look_at_rays(cams[c], (0, 0, 0), args.res, args.res, tile=(4, 8))
        pick = rng.integers(0, o.shape[0], size=int((ci == c).sum()))
        ro_l.append(o[pick]); rd_l.append(d[pick])
    ro, rd = np.concatenate(ro_l), np.concatenate(rd_l)
    gf, gd, go = synth.upstream_grads(ro.shape[0], sc.features.shape[1], seed=7)

    def step():
        oracle.trace(sc, ro, rd, p, margins=None)
        oracle.trace_grad(sc, ro, rd, gf, gd, go, p)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = ro.shape[0] * args.steps / dt / 1e6
    sample = (f"{ro.shape[0]} camera rays per step (random pixels of the workload's cameras), "
              f"forward + gradient, FP64 brute force over {sc.n} surfels")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded object scene and camera rays)",
            "config": {"workload": WORKLOAD, "surfels": sc.n, "rays_per_step": int(ro.shape[0]),
                       "k": 16, "feat_count": int(sc.features.shape[1])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.serve_only:
        import torch
        print(json.dumps({"serving": serve_leg(args, torch.device("cuda", 0))}), flush=True)
        return
    if args.mc_only:
        import torch
        print(json.dumps({"mc": mc_leg(args, torch.device("cuda", 0))}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
