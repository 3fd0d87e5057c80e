"""GB300 differentiable 2D Gaussian ray tracer (IRGS, arXiv 2412.15867).

Thin Python binding over the C ABI of libirgs.so (include/irgs.h). Every step
of the path runs in the library's CUDA kernels; this module only marshals
torch tensors (device memory) and the current CUDA stream into the calls.

    scene = Scene(means, quats, scales, opacity, features, alpha_min=1/255)
    feat, depth, opac = trace(scene, ray_o, ray_d, TraceParams(k=16, feat_count=10))
    (feat.sum() + depth.sum()).backward()      # gradients into the surfel tensors
    rgb = shade_mc(scene, x, n, albedo, rough, wo, env, 32, 32, seed, params)
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, replace

import torch

from . import _lib
from ._lib import IrgsError

__all__ = ["TraceParams", "Scene", "trace", "trace_forward", "trace_backward", "shade_mc",
           "shade_mc_backward", "shade", "EnvMap", "relight", "rasterize", "IrgsError", "library_path"]


FLAG_PER_THREAD = 1   # one traversal stack per ray
FLAG_WARP = 2         # one traversal stack per warp of 32 rays
FLAG_UNIFORM = 4      # shading: stratified uniform hemisphere estimator (Eq. 15)


def library_path() -> str:
    return _lib.LIB_PATH


@dataclass(frozen=True)
class TraceParams:
    """Parameters of a trace (irgs_trace_params)."""
    k: int = 16
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    t_min: float = 0.0
    t_max: float = math.inf
    feat_offset: int = 0
    feat_count: int = 3
    flags: int = 0          # FLAG_PER_THREAD / FLAG_WARP traversal policy (0: library default)

    def c(self) -> _lib.TraceParamsC:
        return _lib.TraceParamsC(int(self.k), float(self.alpha_min), float(self.alpha_max),
                                 float(self.T_min), float(self.t_min), float(self.t_max),
                                 int(self.feat_offset), int(self.feat_count), int(self.flags))

    def with_(self, **kw) -> "TraceParams":
        return replace(self, **kw)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(device) -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev_f32(t: torch.Tensor, name: str, shape_last=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32, got {t.dtype}")
    if shape_last is not None and (t.dim() < 1 or t.shape[-1] != shape_last):
        raise ValueError(f"{name} must have last dimension {shape_last}, got {tuple(t.shape)}")
    return t.contiguous()


class Scene:
    """A resident scene: Morton-ordered surfel copy + LBVH built on the GPU.

    The tensors it was built from are kept so that `trace` can route
    gradients to them; the library itself only keeps its own copies."""

    HIERARCHIES = {"clustered": 0, "radix": 1}   # IRGS_BUILD_RADIX_TREE = 1

    def __init__(self, means, quats, scales, opacity, features=None, alpha_min: float = 1.0 / 255.0,
                 hierarchy: str = "clustered"):
        self.means = _dev_f32(means, "means", 3)
        n = self.means.shape[0]
        self.quats = _dev_f32(quats, "quats", 4)
        self.scales = _dev_f32(scales, "scales", 2)
        self.opacity = _dev_f32(opacity, "opacity").reshape(n)
        if features is None:
            features = torch.zeros((n, 0), device=self.means.device, dtype=torch.float32)
        self.features = _dev_f32(features, "features")
        if self.features.dim() == 1:
            self.features = self.features.reshape(n, 1)
        for name, t in (("quats", self.quats), ("scales", self.scales), ("features", self.features)):
            if t.shape[0] != n:
                raise ValueError(f"{name} has {t.shape[0]} rows, means has {n}")
        if hierarchy not in self.HIERARCHIES:
            raise ValueError(f"hierarchy must be one of {sorted(self.HIERARCHIES)}")
        self.device = self.means.device
        self.alpha_min = float(alpha_min)
        self.hierarchy = hierarchy
        self.num_features = int(self.features.shape[1])
        self.n = int(n)
        L = _lib.lib()
        s = self._surfels()
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(L.irgs_build_scene_ex(C.byref(s), self.alpha_min, self.HIERARCHIES[hierarchy],
                                             _stream(self.device), C.byref(h)), "irgs_build_scene_ex")
        self._h = h

    def _surfels(self) -> _lib.Surfels:
        n = self.n
        return _lib.Surfels(self.means.data_ptr() if n else None, self.quats.data_ptr() if n else None,
                            self.scales.data_ptr() if n else None, self.opacity.data_ptr() if n else None,
                            self.features.data_ptr() if (n and self.num_features) else None,
                            n, self.num_features)

    def _replace(self, means, quats, scales, opacity, features):
        for name, t in (("means", means), ("quats", quats), ("scales", scales), ("opacity", opacity),
                        ("features", features)):
            if t is not None:
                t = _dev_f32(t, name)
                if t.numel() != getattr(self, name).numel():
                    raise ValueError(f"{name} must keep its shape")
                setattr(self, name, t.reshape(getattr(self, name).shape))

    def update(self, means=None, quats=None, scales=None, opacity=None, features=None) -> None:
        """Rebuild the BVH in place after the surfel values changed (same count).
        Tensors given here replace the stored ones (same shapes)."""
        self._replace(means, quats, scales, opacity, features)
        s = self._surfels()
        with torch.cuda.device(self.device):
            _lib.check(_lib.lib().irgs_update_scene(self.handle, C.byref(s), _stream(self.device)),
                       "irgs_update_scene")

    def refit(self, means=None, quats=None, scales=None, opacity=None, features=None) -> None:
        """Refit the BVH to changed surfel values, keeping its Morton order and
        topology (cheaper than update; traces stay exact)."""
        self._replace(means, quats, scales, opacity, features)
        s = self._surfels()
        with torch.cuda.device(self.device):
            _lib.check(_lib.lib().irgs_refit_scene(self.handle, C.byref(s), _stream(self.device)),
                       "irgs_refit_scene")

    @property
    def handle(self) -> C.c_void_p:
        if self._h is None:
            raise ValueError("scene is closed")
        return self._h

    def device_bytes(self) -> int:
        b = C.c_int64()
        _lib.check(_lib.lib().irgs_scene_info(self.handle, None, None, None, C.byref(b)), "irgs_scene_info")
        return int(b.value)

    def status(self) -> int:
        """Synchronise and return (and clear) the device error bits."""
        bits = C.c_uint32()
        _lib.lib().irgs_scene_status(self.handle, _stream(self.device), C.byref(bits))
        return int(bits.value)

    def export(self):
        """Host copies of (perm, keys, nodes[max(n-1,1),16], leaf_boxes[n,6])."""
        import numpy as np
        n = self.n
        perm = np.zeros(max(n, 1), np.int32)
        keys = np.zeros(max(n, 1), np.uint32)
        nodes = np.zeros((max(n - 1, 1), 16), np.float32)
        boxes = np.zeros((max(n, 1), 6), np.float32)
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        _lib.check(_lib.lib().irgs_scene_export(self.handle, p(perm), p(keys), p(nodes), p(boxes)),
                   "irgs_scene_export")
        return perm[:n], keys[:n], nodes, boxes[:n]

    def export_wide(self):
        """Host copy of the 4-wide hierarchy: float32 [n_wide, 32] (see
        irgs_scene_export_wide for the layout)."""
        import numpy as np
        nw = C.c_int64()
        _lib.check(_lib.lib().irgs_scene_export_wide(self.handle, None, 0, C.byref(nw)), "irgs_scene_export_wide")
        out = np.zeros((max(nw.value, 1), 32), np.float32)
        _lib.check(_lib.lib().irgs_scene_export_wide(self.handle, out.ctypes.data_as(C.c_void_p), out.shape[0],
                                                     C.byref(nw)), "irgs_scene_export_wide")
        return out[:nw.value]

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            _lib.lib().irgs_destroy_scene(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rays(scene: Scene, ray_o, ray_d):
    o = _dev_f32(ray_o, "ray_o", 3).reshape(-1, 3)
    d = _dev_f32(ray_d, "ray_d", 3).reshape(-1, 3)
    if o.shape != d.shape:
        raise ValueError("ray_o and ray_d must have the same shape")
    return o, d


def trace_forward(scene: Scene, ray_o, ray_d, params: TraceParams = TraceParams(), max_hit_ids: int = 0,
                  out=None):
    """Forward trace (Eq. 8). Returns dict feat [R,Fc], depth [R], opacity [R],
    n_hits [R] int32 and, if max_hit_ids > 0, hit_ids [R,max_hit_ids] (user
    indices in blend order, -1 after the last one when it fits; a fresh
    array is -1 filled). trace_backward uses hit_ids when present."""
    o, d = _rays(scene, ray_o, ray_d)
    R = o.shape[0]
    dev = scene.device
    if out is None:
        out = {"feat": torch.empty((R, params.feat_count), device=dev, dtype=torch.float32),
               "depth": torch.empty(R, device=dev, dtype=torch.float32),
               "opacity": torch.empty(R, device=dev, dtype=torch.float32),
               "n_hits": torch.empty(R, device=dev, dtype=torch.int32)}
    ids = out.get("hit_ids") if max_hit_ids > 0 else None
    if max_hit_ids > 0 and ids is None:
        ids = torch.full((R, max_hit_ids), -1, device=dev, dtype=torch.int32)
        out["hit_ids"] = ids
    p = params.c()
    with torch.cuda.device(dev):
        _lib.check(_lib.lib().irgs_trace_forward(
            scene.handle, _ptr(o), _ptr(d), R, C.byref(p), _ptr(out["feat"]), _ptr(out["depth"]),
            _ptr(out["opacity"]), _ptr(out["n_hits"]), _ptr(ids), int(max_hit_ids), _stream(dev)),
            "irgs_trace_forward")
    return out


def trace_stats(scene: Scene, ray_o, ray_d, params: TraceParams = TraceParams()):
    """Per-ray traversal counters [R, 4] int32: rounds, node fetches, surfel
    tests, k-buffer insertions (diagnostic run of the forward march)."""
    o, d = _rays(scene, ray_o, ray_d)
    R = o.shape[0]
    out = torch.empty((R, 4), device=scene.device, dtype=torch.int32)
    p = params.c()
    with torch.cuda.device(scene.device):
        _lib.check(_lib.lib().irgs_trace_stats(scene.handle, _ptr(o), _ptr(d), R, C.byref(p), _ptr(out),
                                               _stream(scene.device)), "irgs_trace_stats")
    return out


def trace_backward(scene: Scene, ray_o, ray_d, params: TraceParams, fwd: dict, g_feat, g_depth=None,
                   g_opacity=None, grads=None):
    """Backward of trace_forward; returns (or accumulates into) a dict of
    user-order gradients means/quats/scales/opacity/features. If fwd holds
    hit_ids, rays whose whole hit list is there skip the traversal."""
    o, d = _rays(scene, ray_o, ray_d)
    R = o.shape[0]
    dev = scene.device
    n = scene.n
    if grads is None:
        grads = {"means": torch.zeros((n, 3), device=dev), "quats": torch.zeros((n, 4), device=dev),
                 "scales": torch.zeros((n, 2), device=dev), "opacity": torch.zeros(n, device=dev),
                 "features": torch.zeros((n, scene.num_features), device=dev)}
    gf = _dev_f32(g_feat, "g_feat").reshape(R, params.feat_count)
    ids = fwd.get("hit_ids")
    if ids is not None and (ids.dtype != torch.int32 or ids.dim() != 2 or ids.shape[0] != R
                            or not ids.is_contiguous()):
        raise ValueError("hit_ids must be a contiguous int32 [R, max_hit_ids] tensor")
    gd = None if g_depth is None else _dev_f32(g_depth, "g_depth").reshape(R)
    go = None if g_opacity is None else _dev_f32(g_opacity, "g_opacity").reshape(R)
    p = params.c()
    with torch.cuda.device(dev):
        _lib.check(_lib.lib().irgs_trace_backward(
            scene.handle, _ptr(o), _ptr(d), R, C.byref(p), _ptr(fwd["feat"]), _ptr(fwd["depth"]),
            _ptr(fwd["opacity"]), _ptr(fwd["n_hits"]), _ptr(ids), int(ids.shape[1]) if ids is not None else 0,
            _ptr(gf), _ptr(gd), _ptr(go),
            _ptr(grads["means"]), _ptr(grads["quats"]), _ptr(grads["scales"]), _ptr(grads["opacity"]),
            _ptr(grads["features"]) if scene.num_features else None, _stream(dev)),
            "irgs_trace_backward")
    return grads


class _TraceFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, quats, scales, opacity, features, ray_o, ray_d, scene, params, max_saved_hits):
        out = trace_forward(scene, ray_o, ray_d, params, max_hit_ids=max_saved_hits)
        ctx.scene, ctx.params = scene, params
        ctx.hit_ids = out.get("hit_ids")
        ctx.save_for_backward(ray_o, ray_d, out["feat"], out["depth"], out["opacity"], out["n_hits"])
        ctx.mark_non_differentiable(out["n_hits"])
        return out["feat"], out["depth"], out["opacity"], out["n_hits"]

    @staticmethod
    def backward(ctx, g_feat, g_depth, g_opac, _g_nh):
        ro, rd, feat, depth, opac, nh = ctx.saved_tensors
        scene, params = ctx.scene, ctx.params
        R = ro.reshape(-1, 3).shape[0]
        dev = scene.device
        zf = lambda: torch.zeros((R, params.feat_count), device=dev)
        g_feat = zf() if g_feat is None else g_feat
        fwd = {"feat": feat, "depth": depth, "opacity": opac, "n_hits": nh}
        if ctx.hit_ids is not None:
            fwd["hit_ids"] = ctx.hit_ids
        g = trace_backward(scene, ro, rd, params, fwd, g_feat, g_depth, g_opac)
        ctx.hit_ids = None
        return (g["means"], g["quats"], g["scales"], g["opacity"].reshape(scene.opacity.shape),
                g["features"], None, None, None, None, None)


def trace(scene: Scene, ray_o, ray_d, params: TraceParams = TraceParams(), max_saved_hits: int = 0):
    """Differentiable Trace(r_o, r_d): returns (feat, depth, opacity, n_hits);
    gradients flow to the tensors the scene was built from. With
    max_saved_hits > 0 the forward keeps each ray's hit list (4 bytes per
    entry) and the backward skips the traversal for rays that fit in it."""
    return _TraceFn.apply(scene.means, scene.quats, scene.scales, scene.opacity, scene.features,
                          ray_o, ray_d, scene, params, int(max_saved_hits))


def _shade_params(params: TraceParams, mode: str) -> TraceParams:
    if mode not in ("split", "uniform"):
        raise ValueError("mode must be 'split' or 'uniform'")
    flags = params.flags & ~FLAG_UNIFORM
    return params.with_(flags=flags | (FLAG_UNIFORM if mode == "uniform" else 0))


def _gbuffer(x, n, albedo, rough, wo, env):
    x = _dev_f32(x, "x", 3).reshape(-1, 3)
    P = x.shape[0]
    n = _dev_f32(n, "n", 3).reshape(P, 3)
    albedo = _dev_f32(albedo, "albedo", 3).reshape(P, 3)
    rough = _dev_f32(rough, "rough").reshape(P)
    wo = _dev_f32(wo, "wo", 3).reshape(P, 3)
    env = _dev_f32(env, "env", 3)
    if env.dim() != 3:
        raise ValueError("env must be [H, W, 3]")
    return x, n, albedo, rough, wo, env


def shade_mc(scene: Scene, x, n, albedo, rough, wo, env, n_diffuse: int, n_spec: int, seed: int,
             params: TraceParams, want_aux: bool = False, out=None, mode: str = "split"):
    """Monte Carlo rendering equation per G-buffer point (Eq. 13-15).
    mode "split": n_diffuse cosine + n_spec GGX samples; "uniform":
    n_diffuse stratified uniform directions (n_spec = 0).
    Returns rgb [P,3] (and, with want_aux, vis [P] and ind [P,3])."""
    x, n, albedo, rough, wo, env = _gbuffer(x, n, albedo, rough, wo, env)
    P = x.shape[0]
    dev = scene.device
    if out is None:
        out = {"rgb": torch.empty((P, 3), device=dev)}
        if want_aux:
            out["vis"] = torch.empty(P, device=dev)
            out["ind"] = torch.empty((P, 3), device=dev)
    p = _shade_params(params, mode).c()
    with torch.cuda.device(dev):
        _lib.check(_lib.lib().irgs_shade_mc(
            scene.handle, _ptr(x), _ptr(n), _ptr(albedo), _ptr(rough), _ptr(wo), P, _ptr(env),
            int(env.shape[0]), int(env.shape[1]), int(n_diffuse), int(n_spec),
            C.c_uint64(int(seed) & (2 ** 64 - 1)), C.byref(p), _ptr(out["rgb"]), _ptr(out.get("vis")),
            _ptr(out.get("ind")), _stream(dev)), "irgs_shade_mc")
    return out


def shade_mc_backward(scene: Scene, x, n, albedo, rough, wo, env, n_diffuse: int, n_spec: int, seed: int,
                      params: TraceParams, g_rgb, mode: str = "split", want_env: bool = True, grads=None):
    """Gradient of shade_mc for L = sum g_rgb . rgb with the sample directions
    held fixed. Returns (or accumulates into) a dict albedo [P,3], rough [P],
    env [H,W,3] (if want_env) and the user-order surfel gradients
    means/quats/scales/opacity/features."""
    x, n, albedo, rough, wo, env = _gbuffer(x, n, albedo, rough, wo, env)
    P = x.shape[0]
    dev = scene.device
    ns = scene.n
    if grads is None:
        grads = {"albedo": torch.zeros((P, 3), device=dev), "rough": torch.zeros(P, device=dev),
                 "means": torch.zeros((ns, 3), device=dev), "quats": torch.zeros((ns, 4), device=dev),
                 "scales": torch.zeros((ns, 2), device=dev), "opacity": torch.zeros(ns, device=dev),
                 "features": torch.zeros((ns, scene.num_features), device=dev)}
        if want_env:
            grads["env"] = torch.zeros(env.shape, device=dev)
    g = _dev_f32(g_rgb, "g_rgb", 3).reshape(P, 3)
    p = _shade_params(params, mode).c()
    with torch.cuda.device(dev):
        _lib.check(_lib.lib().irgs_shade_mc_backward(
            scene.handle, _ptr(x), _ptr(n), _ptr(albedo), _ptr(rough), _ptr(wo), P, _ptr(env),
            int(env.shape[0]), int(env.shape[1]), int(n_diffuse), int(n_spec),
            C.c_uint64(int(seed) & (2 ** 64 - 1)), C.byref(p), _ptr(g), _ptr(grads["albedo"]),
            _ptr(grads["rough"]), _ptr(grads.get("env")), _ptr(grads["means"]), _ptr(grads["quats"]),
            _ptr(grads["scales"]), _ptr(grads["opacity"]),
            _ptr(grads["features"]) if scene.num_features else None, _stream(dev)),
            "irgs_shade_mc_backward")
    return grads


def shade_sample_rays(n, rough, wo, n_diffuse: int, n_spec: int, seed: int, mode: str = "split"):
    """Directions [P * S, 3] and validity [P * S] (int32) of the secondary
    rays shade_mc draws for points with normals n, roughness rough and
    outgoing directions wo (ray i = p * S + s, origin x[p])."""
    nn = _dev_f32(n, "n", 3)
    P = nn.shape[0]
    r = _dev_f32(rough, "rough").reshape(P)
    w = _dev_f32(wo, "wo", 3)
    S = n_diffuse + n_spec
    d = torch.empty((P * S, 3), device=nn.device, dtype=torch.float32)
    v = torch.empty(P * S, device=nn.device, dtype=torch.int32)
    flags = FLAG_UNIFORM if mode == "uniform" else 0
    with torch.cuda.device(nn.device):
        _lib.check(_lib.lib().irgs_shade_sample_rays(_ptr(nn), _ptr(r), _ptr(w), P, n_diffuse, n_spec,
                                                     C.c_uint64(seed & (2 ** 64 - 1)), flags, _ptr(d), _ptr(v),
                                                     _stream(nn.device)), "irgs_shade_sample_rays")
    return d, v


class _ShadeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, quats, scales, opacity, features, albedo, rough, env, x, n, wo, scene, cfg):
        nd, ns, seed, params, mode = cfg
        out = shade_mc(scene, x, n, albedo, rough, wo, env, nd, ns, seed, params, mode=mode)
        ctx.scene, ctx.cfg = scene, cfg
        ctx.save_for_backward(albedo, rough, env, x, n, wo)
        return out["rgb"]

    @staticmethod
    def backward(ctx, g_rgb):
        albedo, rough, env, x, n, wo = ctx.saved_tensors
        nd, ns, seed, params, mode = ctx.cfg
        scene = ctx.scene
        g = shade_mc_backward(scene, x, n, albedo, rough, wo, env, nd, ns, seed, params, g_rgb.contiguous(),
                              mode=mode, want_env=ctx.needs_input_grad[7])
        return (g["means"], g["quats"], g["scales"], g["opacity"].reshape(scene.opacity.shape),
                g["features"], g["albedo"].reshape(albedo.shape), g["rough"].reshape(rough.shape),
                g.get("env"), None, None, None, None, None)


def shade(scene: Scene, x, n, albedo, rough, wo, env, n_diffuse: int, n_spec: int, seed: int,
          params: TraceParams, mode: str = "split"):
    """Differentiable shade_mc: returns rgb [P,3]; gradients flow to albedo,
    rough, env and the tensors the scene was built from (directions fixed)."""
    return _ShadeFn.apply(scene.means, scene.quats, scene.scales, scene.opacity, scene.features, albedo, rough,
                          env, x, n, wo, scene, (n_diffuse, n_spec, seed, params, mode))


class EnvMap:
    """Pre-integrated maps of an environment [H,W,3] for the relighting query
    (irradiance, split-sum prefiltered levels, BRDF table, sampling cdfs)."""

    IRR = (32, 64)
    LEVELS = 6
    PREF = (64, 128)
    LUT_N = 32

    def __init__(self, env, device=None):
        env = _dev_f32(env, "env", 3)
        if device is not None:
            env = env.to(device)
        if env.dim() != 3:
            raise ValueError("env must be [H, W, 3]")
        self.device = env.device
        self.H, self.W = int(env.shape[0]), int(env.shape[1])
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(_lib.lib().irgs_envmap_create(_ptr(env), self.H, self.W, _stream(self.device),
                                                     C.byref(h)), "irgs_envmap_create")
        self._h = h

    @property
    def handle(self) -> C.c_void_p:
        if self._h is None:
            raise ValueError("environment map is closed")
        return self._h

    def export(self):
        """Host copies: irr [32,64,3], pref [5,64,128,3], lut [32,32,2],
        row_cdf [H+1] (float64), col_cdf [H,W+1] (float64)."""
        import numpy as np
        out = {"irr": np.zeros(self.IRR + (3,), np.float32),
               "pref": np.zeros((self.LEVELS - 1,) + self.PREF + (3,), np.float32),
               "lut": np.zeros((self.LUT_N, self.LUT_N, 2), np.float32),
               "row_cdf": np.zeros(self.H + 1), "col_cdf": np.zeros((self.H, self.W + 1))}
        with torch.cuda.device(self.device):
            _lib.check(_lib.lib().irgs_envmap_export(self.handle, *(a.ctypes.data_as(C.c_void_p)
                                                                    for a in out.values()), None),
                       "irgs_envmap_export")
            torch.cuda.synchronize(self.device)
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            _lib.lib().irgs_envmap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def relight_sample_rays(envmap: "EnvMap", n_points: int, n_samples: int, seed: int):
    """Directions [P * S, 3], densities [P * S] and validity [P * S] of the
    environment samples relight draws (ray i = p * S + s)."""
    dev = envmap.device
    R = n_points * n_samples
    d = torch.empty((R, 3), device=dev, dtype=torch.float32)
    pdf = torch.empty(R, device=dev, dtype=torch.float32)
    v = torch.empty(R, device=dev, dtype=torch.int32)
    with torch.cuda.device(dev):
        _lib.check(_lib.lib().irgs_relight_sample_rays(envmap.handle, n_points, n_samples,
                                                       C.c_uint64(seed & (2 ** 64 - 1)), _ptr(d), _ptr(pdf),
                                                       _ptr(v), _stream(dev)), "irgs_relight_sample_rays")
    return d, pdf, v


def relight(scene: Scene, envmap: EnvMap, x, n, albedo, rough, wo, n_samples: int, seed: int,
            params: TraceParams, want_aux: bool = False, out=None):
    """Relighting estimate per G-buffer point under `envmap` (supplementary
    relighting details): params.feat_offset / feat_count = 7 select the
    traced [albedo (3), roughness, normal (3)] channels. Returns rgb [P,3]
    (and, with want_aux, vis [P] and ind [P,3])."""
    x = _dev_f32(x, "x", 3).reshape(-1, 3)
    P = x.shape[0]
    n = _dev_f32(n, "n", 3).reshape(P, 3)
    albedo = _dev_f32(albedo, "albedo", 3).reshape(P, 3)
    rough = _dev_f32(rough, "rough").reshape(P)
    wo = _dev_f32(wo, "wo", 3).reshape(P, 3)
    dev = scene.device
    if out is None:
        out = {"rgb": torch.empty((P, 3), device=dev)}
        if want_aux:
            out["vis"] = torch.empty(P, device=dev)
            out["ind"] = torch.empty((P, 3), device=dev)
    p = params.c()
    with torch.cuda.device(dev):
        _lib.check(_lib.lib().irgs_relight(
            scene.handle, envmap.handle, _ptr(x), _ptr(n), _ptr(albedo), _ptr(rough), _ptr(wo), P,
            int(n_samples), C.c_uint64(int(seed) & (2 ** 64 - 1)), C.byref(p), _ptr(out["rgb"]),
            _ptr(out.get("vis")), _ptr(out.get("ind")), _stream(dev)), "irgs_relight")
    return out


def rasterize(scene: Scene, cam, params: TraceParams = TraceParams(), out=None):
    """2D Gaussian rasterisation of the camera's width x height image
    (row-major; `cam` is a serve.Camera, its tile fields ignored): surfels
    with centre view depth > params.t_min blended in centre-depth order
    with the 2DGS screen-space filter. Returns feat [P,Fc], depth [P],
    opacity [P], n_hits [P]."""
    P = int(cam.width) * int(cam.height)
    dev = scene.device
    if out is None:
        out = {"feat": torch.empty((P, params.feat_count), device=dev), "depth": torch.empty(P, device=dev),
               "opacity": torch.empty(P, device=dev), "n_hits": torch.empty(P, device=dev, dtype=torch.int32)}
    p = params.c()
    with torch.cuda.device(dev):
        _lib.check(_lib.lib().irgs_rasterize(
            scene.handle, C.cast(C.pointer(cam), C.c_void_p), C.byref(p), _ptr(out["feat"]), _ptr(out["depth"]),
            _ptr(out["opacity"]), _ptr(out.get("n_hits")), _stream(dev)), "irgs_rasterize")
    return out
