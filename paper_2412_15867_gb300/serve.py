"""Continuous-batching server over resident scenes (host scheduler).

Requests (render: camera rays -> Trace, Eq. 8; relight: camera rays ->
material G-buffer -> Monte Carlo rendering equation, Eq. 13-15) are admitted
while device memory allows, and every scheduling step packs tiles of all
admitted requests -- possibly of different scenes, resolutions and sample
counts -- into one persistent launch of the library's serving kernel
(`irgs_server_step`, replayed from a CUDA graph). Requests that arrive while
others are running join at the next step; a relight request moves from its
G-buffer phase to its shading phase between steps. Each request's results
depend only on that request, not on what it shared launches with.

All device work runs in libirgs.so; this module only keeps queues, builds
the tile tables and measures latency.
"""
from __future__ import annotations

import collections
import ctypes as C
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from . import Scene, TraceParams

TILE_RENDER, TILE_GBUFFER, TILE_SHADE = 0, 1, 2
JOB_RENDER, JOB_RELIGHT = 0, 1


class Camera(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("forward", C.c_float * 3), ("right", C.c_float * 3),
                ("up", C.c_float * 3), ("tan_half_fov", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("tile_w", C.c_int32), ("tile_h", C.c_int32)]


class Job(C.Structure):
    _fields_ = [("kind", C.c_int32), ("scene", C.c_int32), ("cam", Camera), ("n_diffuse", C.c_int32),
                ("n_spec", C.c_int32), ("seed", C.c_uint64), ("env", C.c_void_p), ("env_h", C.c_int32),
                ("env_w", C.c_int32), ("feat", C.c_void_p), ("depth", C.c_void_p), ("opacity", C.c_void_p),
                ("gbuffer", C.c_void_p), ("rgb", C.c_void_p), ("ray_o", C.c_void_p), ("ray_d", C.c_void_p)]


# Planar G-buffer of a relight request (16 P floats): name -> (first plane, width)
GBUFFER_LAYOUT = {"x": (0, 3), "n": (3, 3), "albedo": (6, 3), "rough": (9, 1), "wo": (10, 3), "valid": (13, 1),
                  "opacity": (14, 1)}


def gbuffer_views(g: torch.Tensor, P: int) -> dict:
    """Views of a request's planar G-buffer: x, n, albedo, wo [P, 3]; rough,
    valid, opacity [P]."""
    out = {}
    for k, (o, w) in GBUFFER_LAYOUT.items():
        v = g[o * P:(o + w) * P]
        out[k] = v.view(P, 3) if w == 3 else v
    return out


def pack_gbuffer(x, n, albedo, rough, wo, valid=None) -> torch.Tensor:
    """A planar G-buffer (16 P floats, see gbuffer_views) from device arrays."""
    P = x.shape[0]
    g = torch.zeros(16 * P, device=x.device, dtype=torch.float32)
    v = gbuffer_views(g, P)
    v["x"].copy_(x)
    v["n"].copy_(n)
    v["albedo"].copy_(albedo)
    v["rough"].copy_(rough.reshape(P))
    v["wo"].copy_(wo)
    v["valid"].copy_(torch.ones(P, device=x.device) if valid is None else valid.reshape(P))
    v["opacity"].fill_(1.0)
    return g


class Tile(C.Structure):
    _fields_ = [("kind", C.c_int32), ("job", C.c_int32), ("first", C.c_int32), ("count", C.c_int32)]


def _sigs():
    L = _lib.lib()
    P = C.c_void_p
    L.irgs_server_create.restype = C.c_int
    L.irgs_server_create.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                     C.POINTER(_lib.TraceParamsC), C.POINTER(_lib.TraceParamsC), C.POINTER(P)]
    L.irgs_server_staging.restype = C.c_int
    L.irgs_server_staging.argtypes = [P, C.POINTER(C.POINTER(Job)), C.POINTER(C.POINTER(Tile))]
    L.irgs_server_step.restype = C.c_int
    L.irgs_server_step.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P]
    L.irgs_server_destroy.restype = C.c_int
    L.irgs_server_destroy.argtypes = [P]
    L.irgs_camera_rays.restype = C.c_int
    L.irgs_camera_rays.argtypes = [C.POINTER(Camera), C.c_int64, C.c_int64, P, P, P]
    return L


def make_camera(eye, width: int, height: int, target=(0.0, 0.0, 0.0), fov_deg: float = 60.0,
                tile=(4, 8)) -> Camera:
    """Pinhole look-at camera (z up; x up when looking along z)."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up0 = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) <= 0.99 else np.array([1.0, 0.0, 0.0])
    right = np.cross(fwd, up0)
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    tw, th = tile
    if width % tw or height % th:
        tw = th = 1
    c = Camera()
    c.origin[:] = eye.tolist()
    c.forward[:] = fwd.tolist()
    c.right[:] = right.tolist()
    c.up[:] = up.tolist()
    c.tan_half_fov = math.tan(math.radians(fov_deg) / 2)
    c.width, c.height, c.tile_w, c.tile_h = width, height, tw, th
    return c


def camera_rays(cam: Camera, device="cuda:0", first: int = 0, count: int | None = None):
    """The rays a server step traces for pixels [first, first+count)."""
    L = _sigs()
    n = cam.width * cam.height - first if count is None else count
    o = torch.empty((n, 3), device=device)
    d = torch.empty((n, 3), device=device)
    _lib.check(L.irgs_camera_rays(C.byref(cam), first, n, C.c_void_p(o.data_ptr()), C.c_void_p(d.data_ptr()),
                                  C.c_void_p(torch.cuda.current_stream(device).cuda_stream)), "irgs_camera_rays")
    return o, d


def _check_rays(rays, P):
    if rays is None:
        return
    o, d = rays
    for t in (o, d):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                and t.shape == (P, 3)):
            raise ValueError("explicit rays must be contiguous float32 CUDA tensors [width x height, 3]")


@dataclass
class RenderRequest:
    """Render `scene` from a look-at camera at `eye`, or, with `rays` =
    (ray_o, ray_d) device tensors [width x height, 3], along those rays."""
    scene: int
    eye: tuple
    width: int
    height: int
    fov_deg: float = 60.0
    rays: tuple | None = None

    def __post_init__(self):
        _check_rays(self.rays, self.pixels())

    def pixels(self) -> int:
        return self.width * self.height


@dataclass
class RelightRequest:
    """G-buffer of `scene` from the camera at `eye` (or along `rays`), then
    the Monte Carlo rendering equation at its valid pixels with `spp`
    samples. A caller-made planar `gbuffer` of 16 x width x height floats
    (pack_gbuffer, the layout of irgs_job) skips the G-buffer phase."""
    scene: int
    eye: tuple
    width: int
    height: int
    spp: int
    env: torch.Tensor
    seed: int
    fov_deg: float = 60.0
    rays: tuple | None = None
    gbuffer: torch.Tensor | None = None

    def __post_init__(self):
        _check_rays(self.rays, self.pixels())
        g = self.gbuffer
        if g is not None and not (isinstance(g, torch.Tensor) and g.is_cuda and g.dtype == torch.float32
                                  and g.is_contiguous() and g.numel() == 16 * self.pixels()):
            raise ValueError("gbuffer must be a contiguous float32 CUDA tensor of 16 x width x height floats")

    def pixels(self) -> int:
        return self.width * self.height


@dataclass(eq=False)
class Handle:
    request: object
    arrival: float
    out: dict = field(default_factory=dict)
    phase: int = 0            # render: 0 trace; relight: 0 gbuffer, 1 shade; -1 done
    next_px: int = 0          # next pixel / point of the current phase to hand out
    pending: int = 0          # tiles of the current phase still in flight
    admitted: float = -1.0
    done: float = -1.0
    bytes: int = 0
    rays: int = 0
    jid: int = -1

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Server:
    """Continuous-batching scheduler over `scenes` (resident Scene objects)."""

    def __init__(self, scenes, hbm_budget: int = 8 << 30, max_jobs: int = 64, max_tiles: int = 8192,
                 tile_px: int = 4096, step_rays: int = 8 << 20, use_graph: bool = True,
                 material_offset: int = 3, render: TraceParams | None = None,
                 shade: TraceParams | None = None, batching: bool = True):
        self.scenes = list(scenes)
        self.device = self.scenes[0].device
        self.render_p = render or TraceParams(k=16, feat_offset=0, feat_count=10)
        self.shade_p = shade or TraceParams(k=16, feat_offset=0, feat_count=3, t_min=1e-3)
        self.budget = int(hbm_budget)
        self.max_jobs = max_jobs if batching else 1
        self.max_tiles = max_tiles
        self.tile_px = tile_px
        self.step_rays = step_rays
        self.use_graph = use_graph
        self.L = _sigs()
        arr = (C.c_void_p * len(self.scenes))(*[s.handle.value for s in self.scenes])
        h = C.c_void_p()
        rp, sp = self.render_p.c(), self.shade_p.c()
        _lib.check(self.L.irgs_server_create(arr, len(self.scenes), max_jobs, max_tiles, material_offset,
                                             C.byref(rp), C.byref(sp), C.byref(h)), "irgs_server_create")
        self._h = h
        jp, tp = C.POINTER(Job)(), C.POINTER(Tile)()
        _lib.check(self.L.irgs_server_staging(h, C.byref(jp), C.byref(tp)), "irgs_server_staging")
        self.jobs_tab, self.tiles_tab = jp, tp
        self.waiting = collections.deque()
        self.active: list[Handle] = []
        self.finished: list[Handle] = []
        self.used = 0
        self.steps = 0
        self.rays_total = 0
        self.rays_by_kind = {TILE_RENDER: 0, TILE_GBUFFER: 0, TILE_SHADE: 0}
        self.stream = torch.cuda.Stream(self.device)

    # ---- requests
    def submit(self, req, arrival: float | None = None) -> Handle:
        h = Handle(req, time.perf_counter() if arrival is None else arrival)
        P = req.pixels()
        if isinstance(req, RenderRequest):
            h.bytes = P * 4 * (self.render_p.feat_count + 2)
        else:
            h.bytes = P * 4 * (16 + 3)
        if h.bytes > self.budget:
            raise ValueError("request larger than the memory budget")
        self.waiting.append(h)
        return h

    def _admit(self):
        while self.waiting and len(self.active) < self.max_jobs and self.used + self.waiting[0].bytes <= self.budget:
            h = self.waiting.popleft()
            req = h.request
            P = req.pixels()
            dev = self.device
            with torch.cuda.stream(self.stream):
                if isinstance(req, RenderRequest):
                    h.out = {"feat": torch.empty((P, self.render_p.feat_count), device=dev),
                             "depth": torch.empty(P, device=dev), "opacity": torch.empty(P, device=dev)}
                elif req.gbuffer is not None:
                    h.out = {"gbuffer": req.gbuffer, "rgb": torch.empty((P, 3), device=dev)}
                    h.phase = 1
                else:
                    h.out = {"gbuffer": torch.empty(16 * P, device=dev), "rgb": torch.empty((P, 3), device=dev)}
            h.admitted = time.perf_counter()
            self.used += h.bytes
            self.active.append(h)

    @staticmethod
    def _remaining_rays(h: Handle) -> int:
        req = h.request
        P = req.pixels()
        if isinstance(req, RenderRequest):
            return P - h.next_px
        if h.phase == 0:
            return (P - h.next_px) + P * max(1, req.spp)
        return (P - h.next_px) * max(1, req.spp)

    def _job_struct(self, h: Handle, j: Job):
        req = h.request
        j.kind = JOB_RENDER if isinstance(req, RenderRequest) else JOB_RELIGHT
        j.scene = req.scene
        j.cam = make_camera(req.eye, req.width, req.height, fov_deg=req.fov_deg)
        ptr = lambda t: t.data_ptr() if t is not None else None
        j.ray_o, j.ray_d = (ptr(req.rays[0]), ptr(req.rays[1])) if req.rays is not None else (None, None)
        if j.kind == JOB_RENDER:
            j.feat, j.depth, j.opacity = ptr(h.out["feat"]), ptr(h.out["depth"]), ptr(h.out["opacity"])
            j.gbuffer = j.rgb = j.env = None
            j.n_diffuse = j.n_spec = 0
        else:
            j.gbuffer, j.rgb = ptr(h.out["gbuffer"]), ptr(h.out["rgb"])
            j.feat = j.depth = j.opacity = None
            j.n_diffuse = (req.spp + 1) // 2
            j.n_spec = req.spp // 2
            j.seed = req.seed & (2 ** 64 - 1)
            j.env, j.env_h, j.env_w = ptr(req.env), req.env.shape[0], req.env.shape[1]

    # ---- one scheduling step
    def step(self) -> bool:
        """Admit what fits, run one step over the tiles of the active
        requests (the oldest first with up to a quarter of step_rays, then
        shortest remaining work first, up to step_rays rays in all), retire
        finished requests. Returns False if there was nothing to do."""
        self._admit()
        if not self.active:
            return False
        n_jobs = 0
        n_tiles = 0
        budget = self.step_rays
        plan = []
        # shortest remaining work first: small requests finish in the step
        # they join, large ones take what is left of the ray budget; the
        # oldest request always gets a share, so a stream of small requests
        # cannot starve a large one
        order = sorted(self.active, key=self._remaining_rays)
        oldest = min(self.active, key=lambda h: h.arrival)
        order.remove(oldest)
        order.insert(0, oldest)
        for h in order:
            cap = self.step_rays // 4 if h is oldest and len(order) > 1 else budget
            req = h.request
            P = req.pixels()
            if h.phase < 0:
                continue
            if isinstance(req, RenderRequest) or h.phase == 0:
                kind = TILE_RENDER if isinstance(req, RenderRequest) else TILE_GBUFFER
                per_tile, rays_per_unit = self.tile_px, 1
            else:
                kind = TILE_SHADE
                rays_per_unit = max(1, req.spp)
                per_tile = max(4, self.tile_px // rays_per_unit)
            if h.next_px >= P:
                continue          # phase fully handed out in an earlier step of this loop (cannot happen)
            h.jid = n_jobs
            self._job_struct(h, self.jobs_tab[n_jobs])
            n_jobs += 1
            took = 0
            while h.next_px < P and n_tiles < self.max_tiles and budget > 0 and took < cap:
                cnt = min(per_tile, P - h.next_px)
                t = self.tiles_tab[n_tiles]
                t.kind, t.job, t.first, t.count = kind, h.jid, h.next_px, cnt
                n_tiles += 1
                h.next_px += cnt
                rays = cnt * rays_per_unit
                h.rays += rays
                took += rays
                budget -= rays
                self.rays_total += rays
                self.rays_by_kind[kind] += rays
            plan.append(h)
            if n_tiles >= self.max_tiles or budget <= 0 or n_jobs >= self.max_jobs:
                break
        if n_tiles == 0:
            return False
        _lib.check(self.L.irgs_server_step(self._h, n_jobs, n_tiles, 1 if self.use_graph else 0,
                                           C.c_void_p(self.stream.cuda_stream)), "irgs_server_step")
        self.stream.synchronize()
        self.steps += 1
        now = time.perf_counter()
        still = []
        for h in self.active:
            P = h.request.pixels()
            if h in plan and h.next_px >= P:
                if isinstance(h.request, RelightRequest) and h.phase == 0:
                    h.phase, h.next_px = 1, 0
                    still.append(h)
                    continue
                h.phase = -1
                h.done = now
                self.used -= h.bytes
                self.finished.append(h)
                continue
            still.append(h)
        self.active = still
        return True

    def run_until_idle(self):
        while self.step() or self.waiting:
            pass

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.stream.synchronize()
            self.L.irgs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def latency_stats(handles):
    lat = np.array([h.latency for h in handles]) * 1e3
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max())}


def run_poisson(server: Server, make_request, rate: float, duration: float, warmup: float = 0.0, seed: int = 0):
    """Drive `server` with a Poisson stream of `rate` requests/s for
    warmup + duration seconds (arrival times in real time). Requests that
    arrive during the warm-up are served but not reported. Returns
    (reported handles, wall seconds of the measured window, rays traced in it).
    server.window_stats then holds the window's bounds and how many requests
    (of any arrival time) completed inside it."""
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    t_next = t0 + rng.exponential(1.0 / rate)
    end = t0 + warmup + duration
    measured = []
    rays0 = None
    i = 0
    while True:
        now = time.perf_counter()
        while t_next <= now and t_next < end:
            h = server.submit(make_request(i), arrival=t_next)
            i += 1
            if t_next >= t0 + warmup:
                measured.append(h)
                if rays0 is None:
                    rays0 = server.rays_total
            t_next += rng.exponential(1.0 / rate)
        if not server.step():
            if now >= end and not server.waiting:
                break
            time.sleep(min(0.0005, max(0.0, t_next - time.perf_counter())))
    wall = time.perf_counter() - (t0 + warmup)
    rays = sum(h.rays for h in measured)
    w0, w1 = t0 + warmup, t0 + warmup + duration
    done_in = sum(1 for h in server.finished if w0 <= h.done < w1)
    server.window_stats = {"start": w0, "end": w1, "completed_in_window": done_in}
    return measured, wall, rays
