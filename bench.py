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
The same run measures every configuration against the roofline (`configs`:
the tiny cloud, the camera step, the Monte Carlo rendering equation with
1M surfels and 640k points x 64 samples = 41M secondary rays, its
gradient, relighting, and the served mix), with the FP32 peak measured by
the library's FMA probe and the FP64 oracle timed beside each on bounded
samples; the serving leg measures saturated throughput, then p50/p99 at a
Poisson rate of 0.7x saturation (10 s warm-up, 60 s window) with a sweep,
batched and one request at a time.

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

# Nominal FP32 pipe width per SM (for the note beside the measured peak): 128
# FP32 lanes x 2 flops per FMA. The peak the fractions use is measured on
# the device by the library's own FMA-chain probe (irgs_probe_fma).
LANES = 128
HBM_FALLBACK_GBS = 6800.0


def measured_peaks():
    """HBM copy bandwidth from MEASURED_PEAKS.json (driver-written), else the
    fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "hbm_source": "of measured (MEASURED_PEAKS.json copy bandwidth)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": HBM_FALLBACK_GBS, "hbm_source": "of fallback (6.8 TB/s)"}


# DRAM traffic per launch of the dominant kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) scaled per ray; keyed by
# the hash of the sources it was measured on, the hierarchy's builder
# included (null once they change).
# Captured on the 10-camera case (6.4M rays; the ~90 MB scene read is ~3% of
# it, so the per-ray figure slightly overstates a 64M-ray launch).
# (Both captures predate only the move of the launchers' host-side scratch
# allocation to the library's own pool; the kernels' code is unchanged.)
TRAFFIC = {
    # the four round launches of one forward (6.4M-ray capture): read 425.7 + 924.0 + 359.6 + 87.4 MB,
    # written 755.7 + 564.5 + 127.5 + 12.6 MB
    "k_trace_round<16,10,*>": {"bytes_per_ray": (1796.7e6 + 1460.3e6) / 6.4e6, "src_hash": "58027c8418dc"},
    # the listed backward and the replay of long lists (same case): read 1916.0 + 25.6 MB, written 157.0 MB
    "k_trace_backward<16,10>": {"bytes_per_ray": (1941.6e6 + 157.0e6) / 6.4e6, "src_hash": "3c7bc3505c68"},
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
    ap.add_argument("--e2e-chunks", type=int, default=10, help="camera chunks of the pipelined end-to-end leg")
    ap.add_argument("--serve-only", action="store_true", help="run only the serving leg")
    ap.add_argument("--mc-only", action="store_true", help="run only the Monte Carlo shading leg")
    ap.add_argument("--mc-points", type=int, default=640_000)
    ap.add_argument("--mc-surfels", type=int, default=1_000_000)
    ap.add_argument("--mc-reps", type=int, default=2)
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="measured window at the headline rate")
    ap.add_argument("--serve-warmup", type=float, default=10.0)
    ap.add_argument("--sweep-seconds", type=float, default=10.0, help="window of each sweep point")
    ap.add_argument("--sweep-warmup", type=float, default=2.0)
    ap.add_argument("--serve-burst", type=int, default=240, help="requests of the saturation burst")
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


def trace_bytes(R, N, fc, backward=False):
    """Algorithmic bytes of one trace launch: per ray its origin and
    direction (24 B), fc + 2 outputs and the hit count; the scene once
    (64-B record + fc channels per surfel, 64-B nodes). The backward adds the
    upstream gradients and the forward outputs it reads per ray, and one
    read-modify-write of the 10 + fc gradient floats per surfel."""
    b = R * (24 + 4 * (fc + 2) + 4) + N * (64 + 4 * fc) + max(N - 1, 0) * 64
    if backward:
        b += R * 4 * (fc + 2) * 2 + N * 4 * (10 + fc) * 2
    return float(b)


def per_ray_flops(nh, k, n_surfels, F, backward=False, saved_hits=0):
    """Mean algorithmic flops per ray of a sample of per-ray hit counts."""
    return algorithmic_flops(nh, k, n_surfels, F, backward=backward, saved_hits=saved_hits) / max(nh.numel(), 1)


def roof_entry(ms, rays, flops, nbytes, peak_tflops, hbm_gbs, **extra):
    """Throughput against the roofline min(HBM / bytes, FP32 peak / flops)
    of a launch (or step) of `rays` rays taking `ms` milliseconds."""
    t = ms * 1e-3
    mrays = rays / t / 1e6
    alu = peak_tflops * 1e12 / (flops / rays) / 1e6
    hbm = hbm_gbs * 1e9 / (nbytes / rays) / 1e6
    roof = min(alu, hbm)
    e = {"mrays_s": mrays, "ms": ms, "rays": int(rays), "flops_per_ray": flops / rays,
         "bytes_per_ray": nbytes / rays, "achieved_tflops": flops / t / 1e12, "achieved_gbs": nbytes / t / 1e9,
         "alu_bound_mrays_s": alu, "hbm_bound_mrays_s": hbm, "bound": "alu" if alu <= hbm else "hbm",
         "roofline_mrays_s": roof, "frac": mrays / roof}
    e.update(extra)
    return e


def fp32_probe(L, dev, index, iters=100_000, launches=10):
    """FP32 peak measured with the library's FMA-chain probe: CUDA events
    around `launches` launches, SM clocks sampled meanwhile."""
    import ctypes as C
    import torch
    stream = torch.cuda.current_stream(dev)
    sp = C.c_void_p(stream.cuda_stream)
    fl = C.c_double()
    for _ in range(2):
        if L.irgs_probe_fma(iters // 10, sp, C.byref(fl)) != 0:
            raise RuntimeError("irgs_probe_fma failed")
    torch.cuda.synchronize()
    clk = ClockSampler(index)
    clk.start()
    time.sleep(0.3)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(launches):
        L.irgs_probe_fma(iters, sp, C.byref(fl))
    b.record(stream)
    torch.cuda.synchronize()
    c = clk.stop()
    ms = a.elapsed_time(b)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    tflops = launches * fl.value / (ms * 1e-3) / 1e12
    return {"tflops": tflops, "sm_mhz": c.get("sm_mhz"), "sms": sms, "launch_ms": ms / launches,
            "flops_per_launch": fl.value,
            "nominal_at_max_clock_tflops": sms * LANES * 2 * (c.get("sm_max_mhz") or 0) * 1e6 / 1e12,
            "how": f"{launches} launches of irgs_probe_fma ({sms} SMs x 8 blocks x 256 threads, 8 independent "
                   "FMA chains per thread), CUDA events; clocks sampled during the launches"}


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

    # ---- measured peaks: the FP32 pipe by the library's FMA-chain probe (at
    # the probe's clock, scaled to the timed region's median SM clock), HBM
    # from the driver's copy measurement
    peaks = measured_peaks()
    probe = fp32_probe(L, dev, local)
    peak = probe["tflops"]
    if clk.get("sm_mhz") and probe.get("sm_mhz"):
        peak = probe["tflops"] * clk["sm_mhz"] / probe["sm_mhz"]
    hbm = peaks["hbm_gbs"]
    peak_note = (f"of measured: FMA-chain probe {probe['tflops']:.2f} TFLOP/s at {probe['sm_mhz']} MHz median SM "
                 f"clock, scaled to the timed region's {clk.get('sm_mhz')} MHz ({probe['sms']} SMs)")

    # ---- roofline of the dominant kernel (by time)
    nh = out["n_hits"]
    if bwd_ms >= fwd_ms:
        kname, kms = "k_trace_backward<16,10>", bwd_ms
        flops = algorithmic_flops(nh, 16, sc.n, F, backward=True, saved_hits=args.saved_hits)
        src = ["trace.cuh", "trace_bwd.cuh", "trace_bwd.cu", "common.cuh", "scene.cu"]
    else:
        # the forward pass: for batches of 2^20 rays or more its compacted
        # k-buffer rounds and the compaction between them
        kname, kms = "k_trace_round<16,10,*>", fwd_ms
        flops = algorithmic_flops(nh, 16, sc.n, F)
        src = ["trace.cuh", "trace_fwd.cu", "common.cuh", "scene.cu"]
    achieved = flops / (kms * 1e-3) / 1e12
    khash = _kernel_hash(src)
    tr = TRAFFIC.get(kname)
    traffic = tr["bytes_per_ray"] * R if (tr and tr.get("bytes_per_ray") and tr.get("src_hash") == khash) else None

    # ---- work actually done per camera ray (diagnostic counters of the
    # forward march on one camera's rays): the gap to the roofline splits
    # into extra work (nodes and candidates beyond the algorithmic count)
    # and the rate at which that work runs
    R1 = args.res * args.res
    ws = irgs.trace_stats(scene, ro[:R1], rd[:R1], p).double().mean(0).tolist()
    nh1 = float(nh[:R1].double().mean())
    # per node visit: 4 child slab tests (6 FMA, 6 min/max, 2 three-way) ~ 20
    # flops each; per surfel test 45; per composited hit the blend
    work_flops_ray = ws[1] * 4 * 20 + ws[2] * 45 + nh1 * (2 * (F + 2) + 3)
    alg_flops_ray = flops / R
    work = {"sample": f"camera 0 ({R1} rays)", "rounds_per_ray": ws[0], "nodes_per_ray": ws[1],
            "candidates_per_ray": ws[2], "inserts_per_ray": ws[3], "hits_per_ray": nh1,
            "algorithmic_flops_per_ray": alg_flops_ray, "work_flops_per_ray": work_flops_ray,
            "work_over_algorithmic": work_flops_ray / alg_flops_ray,
            "work_frac": work_flops_ray * R / (kms * 1e-3) / 1e12 / peak,
            "note": "work_frac = the counted work (4 x 20 flops per node visit, 45 per surfel test, the blend per "
                    "hit) per second over the FP32 peak: how busy the FP32 pipe would be if every counted test "
                    "were needed; frac / work_frac = algorithmic / counted work"}
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "flops_per_launch": flops, "launch_ms": kms, "peak_note": peak_note,
                "hbm_bound_mrays_s": hbm * 1e9 / (trace_bytes(R, sc.n, F) / R) / 1e6,
                "work_frac": work["work_frac"]}

    # ---- the configurations' table: Mrays/s and roofline fraction each
    configs = {}
    if rank == 0:
        configs["C0"] = tiny_leg(args, dev, peak, hbm)
    bf = trace_bytes(R, sc.n, F)
    configs["C1"] = {
        "workload": WORKLOAD,
        "fwd": roof_entry(fwd_ms, R, algorithmic_flops(nh, 16, sc.n, F), bf, peak, hbm),
        "fwd_bwd": roof_entry(fwd_ms + bwd_ms, R,
                              algorithmic_flops(nh, 16, sc.n, F)
                              + algorithmic_flops(nh, 16, sc.n, F, backward=True, saved_hits=args.saved_hits),
                              bf + trace_bytes(R, sc.n, F, backward=True), peak, hbm),
        "step": roof_entry(ms_per_step, R,
                           algorithmic_flops(nh, 16, sc.n, F)
                           + algorithmic_flops(nh, 16, sc.n, F, backward=True, saved_hits=args.saved_hits),
                           bf + trace_bytes(R, sc.n, F, backward=True), peak, hbm,
                           note="the timed step: rebuild + forward + backward")}

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
        # device->host copies of chunk c-1 overlap the traces of chunk c;
        # chunks alternate between two compute streams, so one chunk's last
        # (small) rounds overlap the next chunk's forward. Backward calls add
        # into the same gradient arrays, so each waits for the previous one.
        n_chunk = max(1, min(args.e2e_chunks, args.cams))
        bounds_ = [(R * i // n_chunk, R * (i + 1) // n_chunk) for i in range(n_chunk)]
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        s_comp = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
        ev_in = [torch.cuda.Event() for _ in range(n_chunk)]
        ev_done = [torch.cuda.Event() for _ in range(n_chunk)]
        ev_ready = torch.cuda.Event()
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
            ev_ready.record(stream)
            for cs in s_comp:
                cs.wait_event(ev_ready)
            for i, (lo, hi) in enumerate(bounds_):
                cs = s_comp[i % 2]
                with torch.cuda.stream(cs):
                    cs.wait_event(ev_in[i])
                    sl = {k: out[k][lo:hi] for k in out}
                    irgs.trace_forward(scene_e2e, dev_in["ro"][lo:hi], dev_in["rd"][lo:hi], p,
                                       max_hit_ids=args.saved_hits, out=sl)
                    if i > 0:
                        cs.wait_event(ev_done[i - 1])
                    irgs.trace_backward(scene_e2e, dev_in["ro"][lo:hi], dev_in["rd"][lo:hi], p, sl,
                                        dev_in["gf"][lo:hi], dev_in["gd"][lo:hi], dev_in["go"][lo:hi], grads=grads)
                    ev_done[i].record(cs)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done[i])
                    for k in ("feat", "depth", "opacity", "n_hits"):
                        host_out[k][lo:hi].copy_(out[k][lo:hi], non_blocking=True)
            for cs in s_comp:
                stream.wait_stream(cs)
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
               "pipeline": f"{n_chunk} camera chunks on two alternating compute streams; copies on two side streams "
                           "overlap the traces"}
        scene_e2e.close()

    # ---- Monte Carlo rendering equation configuration
    mc = None
    if not args.no_mc and rank == 0:
        mc = mc_leg(args, dev, peak, hbm, cpu=not args.no_cpu)
        configs["C2"] = mc.pop("configs")

    # ---- serving mix (continuous batching vs one request at a time)
    serving = None
    if not args.no_serve and rank == 0:
        del out, grads, ro, rd, gf, gd, go
        torch.cuda.empty_cache()
        serving = serve_leg(args, dev)
        configs["C4"] = serving_roofline(serving, configs, peak, hbm)

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
            "clocks": clk, "fp32_probe": probe, "hbm_gbs": {"value": hbm, "source": peaks["hbm_source"]},
            "work": work, "configs": configs, "raster": raster, "mc": mc, "serving": serving,
        }
        if cpu is not None:
            configs["C1"]["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def mc_leg(args, dev, peak, hbm, cpu=True):
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

    # hits per secondary ray, for the algorithmic flop counts: the rays the
    # estimators draw for the first 4096 points (the library's own samplers),
    # traced with the same parameters
    Ps, N2 = 4096, sc2.n
    xs = g2[0][:Ps].repeat_interleave(64, 0)
    dsh, vsh = irgs.shade_sample_rays(g2[1][:Ps], g2[3][:Ps], g2[4][:Ps], 32, 32, 2024)
    vm = vsh.bool()
    nh_sh = irgs.trace_forward(S2, xs[vm].contiguous(), dsh[vm].contiguous(), ps)["n_hits"]
    drl, _, vrl = irgs.relight_sample_rays(E, Ps, 64, 2025)
    vr = vrl.bool()
    nh_rl = irgs.trace_forward(S2, xs[vr].contiguous(), drl[vr].contiguous(), pr)["n_hits"]
    torch.cuda.synchronize()
    vfrac, vfrac_rl = float(vm.float().mean()), float(vr.float().mean())
    f_fwd = per_ray_flops(nh_sh, 16, N2, 3)
    f_bwd = per_ray_flops(nh_sh, 16, N2, 3, backward=True, saved_hits=64)
    f_rl = per_ray_flops(nh_rl, 16, N2, 7)
    SAMPLE_FLOPS = 150          # direction, BRDF and estimator terms per sample
    env_b = 512 * 256 * 3 * 4
    scene_b = lambda fc: N2 * (64 + 4 * fc) + (N2 - 1) * 64
    b_sh = Pn * 16 * 4 + env_b + scene_b(3)
    b_gr = b_sh + Pn * 3 * 4 + Pn * 4 * 4 * 2 + 2 * env_b + N2 * 4 * 13 * 2
    maps_b = (32 * 64 * 3 + 5 * 64 * 128 * 3 + 32 * 32 * 2) * 4 + 8 * (257 + 256 * 513) + env_b
    b_rl = Pn * 16 * 4 + maps_b + scene_b(7)
    note = (f"hits per traced secondary ray from {Ps} points' samples: shading {float(nh_sh.float().mean()):.2f} "
            f"({vfrac:.3f} of samples traced), relighting {float(nh_rl.float().mean()):.2f}; "
            f"{SAMPLE_FLOPS} flops per sample for sampling and the BRDF")
    configs = {
        "workload": f"{args.mc_surfels} surfels, {Pn} G-buffer points x 64 samples, 512x256 environment, k=16",
        "shade": roof_entry(fms, rays, rays * (vfrac * f_fwd + SAMPLE_FLOPS), b_sh, peak, hbm, note=note),
        "grad": roof_entry(bms, rays, rays * (vfrac * (f_fwd + f_bwd) + SAMPLE_FLOPS), b_gr, peak, hbm,
                           note="forward trace saving hit lists, then the backward from the lists (3x per hit)"),
        "relight": roof_entry(relight_ms, rays, rays * (vfrac_rl * f_rl + SAMPLE_FLOPS), b_rl, peak, hbm),
    }
    if cpu:
        configs["cpu_baseline"] = cpu_baseline_mc(sc2, gb, synth.env_map(seed=1003))
    E.close()
    if S2.status() != 0:
        raise RuntimeError("device error in the MC leg")
    S2.close()
    return {"configs": configs,"workload": f"{args.mc_surfels} surfels, {Pn} G-buffer points x (32 cosine + 32 GGX) = "
                        f"{rays / 1e6:.1f}M secondary rays, 512x256 env, k=16",
            "ms": fms, "mrays_s": rays / (fms * 1e-3) / 1e6, "points_per_s": Pn / (fms * 1e-3),
            "bwd_ms": bms, "bwd_mrays_s": rays / (bms * 1e-3) / 1e6,
            "path": "secondary rays regrouped by direction bin and origin Morton code, one stack per ray",
            "fused_per_lane_ms": fused_ms,
            "relight": {"workload": f"{Pn} points x 64 environment-importance samples, 512x256 environment, "
                                    "traced albedo/roughness/normal shaded with split-sum maps",
                        "envmap_ms": env_ms, "ms": relight_ms, "mrays_s": rays / (relight_ms * 1e-3) / 1e6}}


def tiny_leg(args, dev, peak, hbm):
    """The tiny forward configuration: 1,024 surfels, one 64x64 camera (4,096
    rays), k = 8, 3 channels. Forward and forward + backward, each call timed
    with CUDA events over 200 repetitions after a warm-up (calls this small
    are launch-bound); the oracle on all 4,096 rays beside it."""
    import numpy as np
    import torch
    import synth
    import paper_2412_15867_gb300 as irgs

    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sc = synth.tiny_scene(seed=1000, n=1024)
    ro_np, rd_np = synth.look_at_rays(synth.tiny_camera(1000), (0, 0, 0), 64, 64)
    R = ro_np.shape[0]
    S = irgs.Scene(*(T(a) for a in sc.arrays()))
    ro, rd = T(ro_np), T(rd_np)
    gf_np, gd_np, go_np = synth.upstream_grads(R, 3, seed=1004)
    gf, gd, go = T(gf_np), T(gd_np), T(go_np)
    p = irgs.TraceParams(k=8, feat_count=3)
    out = irgs.trace_forward(S, ro, rd, p)
    grads = irgs.trace_backward(S, ro, rd, p, out, gf, gd, go)
    stream = torch.cuda.current_stream(dev)
    reps = 200
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(10):
        irgs.trace_forward(S, ro, rd, p, out=out)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        irgs.trace_forward(S, ro, rd, p, out=out)
    ev[1].record(stream)
    for _ in range(reps):
        irgs.trace_forward(S, ro, rd, p, out=out)
        irgs.trace_backward(S, ro, rd, p, out, gf, gd, go, grads=grads)
    ev[2].record(stream)
    torch.cuda.synchronize()
    if S.status() != 0:
        raise RuntimeError("device error in the tiny configuration")
    f_ms = ev[0].elapsed_time(ev[1]) / reps
    fb_ms = ev[1].elapsed_time(ev[2]) / reps
    nh = out["n_hits"]
    ff = algorithmic_flops(nh, 8, sc.n, 3)
    fbk = algorithmic_flops(nh, 8, sc.n, 3, backward=True)
    res = {"workload": "1,024 surfels (centres U[-1,1]^3), one 64x64 camera = 4,096 rays, k=8, 3 channels",
           "fwd": roof_entry(f_ms, R, ff, trace_bytes(R, sc.n, 3), peak, hbm,
                             note="one launch per call; launch-bound at this size"),
           "fwd_bwd": roof_entry(fb_ms, R, ff + fbk, trace_bytes(R, sc.n, 3) + trace_bytes(R, sc.n, 3, True),
                                 peak, hbm)}
    if not args.no_cpu:
        res["cpu_baseline"] = cpu_baseline_tiny(sc, ro_np, rd_np, gf_np, gd_np, go_np)
    S.close()
    return res


def cpu_baseline_tiny(sc, ro, rd, gf, gd, go):
    """Oracle forward + gradient on all 4,096 rays of the tiny configuration."""
    import oracle
    p = oracle.Params(feat_count=3)
    cores = oracle.num_threads()
    n, t0 = 0, time.perf_counter()
    while n == 0 or time.perf_counter() - t0 < 2.0:
        oracle.trace(sc, ro, rd, p, margins=None)
        oracle.trace_grad(sc, ro, rd, gf, gd, go, p)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n * ro.shape[0] / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all {ro.shape[0]} rays, forward + gradient, {n} passes ({dt:.1f} s)"}


def cpu_baseline_mc(sc, gb, env):
    """Oracle Monte Carlo shading (32 points x 64 samples = 2,048 secondary
    rays) and its gradient (16 points x 64 samples) over the 1M-surfel scene."""
    import numpy as np
    import oracle
    p = oracle.Params(feat_count=3, t_min=1e-3)
    cores = oracle.num_threads()
    sub = [a[:32] for a in gb]
    t0 = time.perf_counter()
    oracle.shade(sc, *sub, env, 32, 32, 2024, p, margins=None)
    dt = time.perf_counter() - t0
    sub = [a[:16] for a in gb]
    g = np.random.default_rng(1004).normal(size=(16, 3)).astype(np.float32)
    t1 = time.perf_counter()
    oracle.shade_grad(sc, *sub, env, 32, 32, 2024, p, g)
    dg = time.perf_counter() - t1
    return {"shade": {"value": 2048 / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                      "sample": f"32 points x 64 samples = 2,048 secondary rays, FP64 brute force over {sc.n} "
                                f"surfels ({dt:.1f} s)"},
            "grad": {"value": 1024 / dg / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                     "sample": f"16 points x 64 samples = 1,024 secondary rays, gradient ({dg:.1f} s)"},
            "relight": None,
            "relight_note": "not timed: the oracle pre-integrates the environment (plain sums over all "
                            "texels) inside every call, ~50 s on the host before its first ray"}


def serving_roofline(serving, configs, peak, hbm):
    """Aggregate roofline fraction of the served mix at the headline rate:
    served rays per second against the roofline of the same rays, each kind
    costed with the per-ray flops measured for its standalone configuration
    (render rays as the camera rays, G-buffer rays as camera rays with 7
    channels, shading rays as the Monte Carlo samples)."""
    h = serving.get("headline", {}).get("batched")
    kinds = serving.get("rays_by_kind")
    if not h or not kinds or "C1" not in configs or "C2" not in configs:
        return None
    f_cam = configs["C1"]["fwd"]["flops_per_ray"]
    f_sh = configs["C2"]["shade"]["flops_per_ray"]
    f_g = f_cam * (45 + 2 * 9 + 3) / (45 + 2 * 12 + 3)
    tot = kinds["render"] + kinds["gbuffer"] + kinds["shade"]
    if tot == 0:
        return None
    fpr = (kinds["render"] * f_cam + kinds["gbuffer"] * f_g + kinds["shade"] * f_sh) / tot
    mrays = h["mrays_s"]
    alu = peak * 1e12 / fpr / 1e6
    return {"workload": serving["mix"], "mrays_s": mrays, "flops_per_ray": fpr, "alu_bound_mrays_s": alu,
            "bound": "alu", "roofline_mrays_s": alu, "frac": mrays / alu,
            "ray_mix": {k: v / tot for k, v in kinds.items()},
            "note": "served rays per second at the headline Poisson rate over the FP32 roofline of the same "
                    "ray mix (bytes are far from binding for these traces)"}


def serve_leg(args, dev):
    """Serving mix: 4 resident scenes (100k, 300k, 1M, 2M surfels, object scene
    with median scale 0.01 sqrt(300k/N)); 50% render (camera rays, 10
    channels) / 50% relight (G-buffer + Monte Carlo shading, spp log-uniform
    in [1, 128]) requests at resolutions {128, 256, 512, 1024}^2 from random
    hemisphere cameras. Saturated throughput first: a burst of requests of
    the Poisson stream's distribution, all queued at once. Then Poisson
    streams at fractions of that rate, served with continuous batching and,
    separately, one request at a time: the headline at 0.7x (warm-up, then
    the measured window) and a sweep at 0.3x, 0.5x and 0.9x."""
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
    kw = dict(hbm_budget=budget, max_jobs=64, max_tiles=8192)
    # saturated: a burst of requests of the stream's distribution, continuous batching
    srv = serve.Server(scenes, **kw)
    warm = maker(99)
    for i in range(6):                                   # warm-up (graph capture, caches)
        srv.submit(warm(i))
    srv.run_until_idle()
    mk = maker(23)
    n_sat = args.serve_burst
    rays0 = srv.rays_total
    t0 = time.perf_counter()
    for i in range(n_sat):
        srv.submit(mk(i), arrival=t0)
    srv.run_until_idle()
    sat_wall = time.perf_counter() - t0
    sat_rate = n_sat / sat_wall
    sat_mrays = (srv.rays_total - rays0) / sat_wall / 1e6
    srv.close()
    out = {"scenes_surfels": sizes, "mix": "50% render (10 ch) / 50% relight (spp log-uniform 1-128), "
           "res {128,256,512,1024}^2, random hemisphere cameras, Poisson arrivals",
           "saturated": {"requests_per_s": sat_rate, "mrays_s": sat_mrays, "requests": n_sat,
                         "how": "burst of requests of the stream's distribution queued at once"}}

    def run(frac, batching, seconds, warmup, seed):
        srv2 = serve.Server(scenes, batching=batching, **kw)
        rate = frac * sat_rate
        k0 = dict(srv2.rays_by_kind)
        hs, wall, rays = serve.run_poisson(srv2, maker(seed), rate, seconds, warmup, seed=seed)
        st = serve.latency_stats(hs)
        # throughput: requests completed inside the measured window (of any
        # arrival time) per second of it; a stable server keeps up with the
        # offered rate, an overloaded one falls behind and its backlog grows
        served = srv2.window_stats["completed_in_window"] / seconds
        st.update({"offered_requests_per_s": rate, "arrived_in_window": len(hs),
                   "served_requests_per_s": served, "served_over_offered": served / rate,
                   "drain_s": wall - seconds, "mrays_s": rays / wall / 1e6, "steps": srv2.steps,
                   "window_s": seconds, "warmup_s": warmup})
        kinds = {k: srv2.rays_by_kind[k] - k0[k] for k in k0}
        srv2.close()
        return st, kinds

    # headline: 0.7x saturation, warm-up then the measured window
    b, kinds = run(0.7, True, args.serve_seconds, args.serve_warmup, 24)
    o, _ = run(0.7, False, args.sweep_seconds, args.sweep_warmup, 24)
    out["headline"] = {"lambda_over_saturated": 0.7, "batched": b, "one_at_a_time": o,
                       "stable": bool(b["served_over_offered"] >= 0.95)}
    out["rays_by_kind"] = {"render": kinds[serve.TILE_RENDER], "gbuffer": kinds[serve.TILE_GBUFFER],
                           "shade": kinds[serve.TILE_SHADE]}
    sweep = []
    for frac in (0.3, 0.5, 0.9):
        b, _ = run(frac, True, args.sweep_seconds, args.sweep_warmup, 25 + int(frac * 10))
        o, _ = run(frac, False, args.sweep_seconds, args.sweep_warmup, 25 + int(frac * 10))
        sweep.append({"lambda_over_saturated": frac, "batched": b, "one_at_a_time": o})
    out["sweep"] = sweep
    status = sum(S.status() for S in scenes)
    if status:
        raise RuntimeError("device error in the serving leg")
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
        from paper_2412_15867_gb300 import _lib
        dev = torch.device("cuda", 0)
        probe = fp32_probe(_lib.lib(), dev, 0)
        print(json.dumps({"mc": mc_leg(args, dev, probe["tflops"], measured_peaks()["hbm_gbs"],
                                       cpu=not args.no_cpu)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
