"""FP64 CPU oracle for the 2D Gaussian ray tracer -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference legs
of `bench.py` may import this package. The product path (the CUDA library and
its Python binding) never does, and never falls back to it.

The arithmetic lives in `irgs_oracle.c` (plain C, FP64, OpenMP over rays);
this module compiles it with gcc and wraps it with ctypes. Inputs are the
float32 arrays produced by `synth`; outputs are float64 NumPy arrays.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "irgs_oracle.c")
_OBJ = os.path.join(_HERE, "_obj")
_LIB_PATH = os.path.join(_OBJ, "libirgs_oracle.so")
_lock = threading.Lock()
_lib = None

# ambiguity flag bits (must match irgs_oracle.c)
F_ALPHA, F_RHO, F_T, F_TIE, F_TRANGE, F_GRAZE, F_CLAMP = 1, 2, 4, 8, 16, 32, 64
FORWARD_FLAGS = F_ALPHA | F_RHO | F_T | F_TIE | F_TRANGE | F_GRAZE


class _Params(C.Structure):
    _fields_ = [("alpha_min", C.c_double), ("alpha_max", C.c_double), ("T_min", C.c_double),
                ("t_min", C.c_double), ("t_max", C.c_double),
                ("feat_offset", C.c_int32), ("feat_count", C.c_int32)]


class _Margins(C.Structure):
    _fields_ = [("alpha_abs", C.c_double), ("rho_rel", C.c_double), ("T_rel", C.c_double),
                ("tie_abs", C.c_double), ("t_abs", C.c_double), ("clamp_abs", C.c_double)]


@dataclass
class Params:
    """Trace parameters (see the readings in irgs_oracle.c)."""
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    t_min: float = 0.0
    t_max: float = math.inf
    feat_offset: int = 0
    feat_count: int = 3

    def c(self) -> _Params:
        return _Params(self.alpha_min, self.alpha_max, self.T_min, self.t_min, self.t_max,
                       self.feat_offset, self.feat_count)


@dataclass
class Margins:
    """Margins of the per-ray ambiguity flags."""
    alpha_abs: float = 1e-6
    rho_rel: float = 1e-5
    T_rel: float = 1e-5
    tie_abs: float = 2e-8
    t_abs: float = 1e-6
    clamp_abs: float = 1e-5

    def c(self) -> _Margins:
        return _Margins(self.alpha_abs, self.rho_rel, self.T_rel, self.tie_abs, self.t_abs,
                        self.clamp_abs)


def build(force: bool = False) -> str:
    """Compile irgs_oracle.c into a shared library (gcc, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OBJ, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.oracle_trace.restype = C.c_int
    lib.oracle_trace.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, P, P, C.c_int64,
                                 P, P, P, P, P, P, P, P, C.c_int32, P, C.c_int]
    lib.oracle_trace_alternatives.restype = C.c_int
    lib.oracle_trace_alternatives.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, P, P, C.c_int64,
                                              P, P, C.c_int32, P, P, P, P, P, C.c_int]
    lib.oracle_shade_bounds.restype = C.c_int
    lib.oracle_shade_bounds.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, P, P, P, P, P, C.c_int64,
                                        P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P,
                                        P, P, C.c_int32, P, P, P, C.c_int]
    lib.oracle_relight_bounds.restype = C.c_int
    lib.oracle_relight_bounds.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, P, P, P, P, P, C.c_int64,
                                          P, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P, P, P, C.c_int32,
                                          P, P, P, C.c_int]
    lib.oracle_trace_grad.restype = C.c_int
    lib.oracle_trace_grad.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, P, P, C.c_int64,
                                      P, P, P, P, P, P, P, P, P, C.c_int]
    lib.oracle_shade.restype = C.c_int
    lib.oracle_shade.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, P, P, P, P, P, C.c_int64,
                                 P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P,
                                 P, P, P, P, P, P, C.c_int]
    lib.oracle_shade_grad.restype = C.c_int
    lib.oracle_shade_grad.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, P, P, P, P, P, C.c_int64,
                                      P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P,
                                      P, P, P, P, P, P, P, P, P, P, C.c_int]
    lib.oracle_splitmix64.restype = C.c_uint64
    lib.oracle_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
    lib.oracle_env_lookup.restype = None
    lib.oracle_env_lookup.argtypes = [P, C.c_int32, C.c_int32, P, P]
    lib.oracle_sample_dirs.restype = C.c_int
    lib.oracle_sample_dirs.argtypes = [P, P, P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P, P]
    lib.oracle_num_threads.restype = C.c_int
    lib.oracle_num_threads.argtypes = [C.c_int]
    lib.oracle_rasterize.restype = C.c_int
    lib.oracle_rasterize.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, P, P, P, P, P, P, P, P, C.c_int]
    lib.oracle_relight_maps.restype = C.c_int
    lib.oracle_relight_maps.argtypes = [P, C.c_int32, C.c_int32, C.c_int, P, P, P, P, P]
    lib.oracle_env_samples.restype = C.c_int
    lib.oracle_env_samples.argtypes = [P, C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.c_uint64, P, P]
    lib.oracle_relight.restype = C.c_int
    lib.oracle_relight.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, P, P, P, P, P, C.c_int64,
                                   P, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P, P, P, P, P, P, P, C.c_int]
    _lib = lib
    return lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads(n: int = 0) -> int:
    """OpenMP threads the oracle uses (n > 0 sets it)."""
    return int(_load().oracle_num_threads(int(n)))


def _surfel_arrays(scene):
    means, quats, scales, opacity, feats = (_f32(a) for a in scene.arrays())
    if feats.ndim == 1:
        feats = feats.reshape(-1, 1)
    return means, quats, scales, opacity, feats


def trace(scene, ray_o, ray_d, params: Params = Params(), margins: Margins | None = Margins(),
          max_ids: int = 0, n_threads: int = 0):
    """Brute-force FP64 forward trace (Eq. 8). Returns a dict with feat [R,Fc],
    depth [R], opacity [R], n_hits [R], flags [R] (ambiguity bits) and, if
    max_ids > 0, ids [R,max_ids] / tau [R,max_ids] of the composited hits."""
    lib = _load()
    means, quats, scales, opacity, feats = _surfel_arrays(scene)
    o, d = _f32(ray_o).reshape(-1, 3), _f32(ray_d).reshape(-1, 3)
    R, n, F = o.shape[0], means.shape[0], feats.shape[1]
    fc = params.feat_count
    out = {
        "feat": np.zeros((R, fc), np.float64),
        "depth": np.zeros(R, np.float64),
        "opacity": np.zeros(R, np.float64),
        "n_hits": np.zeros(R, np.int32),
        "flags": np.zeros(R, np.uint32),
    }
    ids = tau = None
    if max_ids > 0:
        ids = np.zeros((R, max_ids), np.int32)
        tau = np.zeros((R, max_ids), np.float64)
    m = margins.c() if margins is not None else None
    p = params.c()
    rc = lib.oracle_trace(_ptr(means), _ptr(quats), _ptr(scales), _ptr(opacity), _ptr(feats),
                          n, F, _ptr(o), _ptr(d), R, C.byref(p),
                          C.byref(m) if m is not None else None,
                          _ptr(out["feat"]), _ptr(out["depth"]), _ptr(out["opacity"]),
                          _ptr(out["n_hits"]), _ptr(ids), _ptr(tau), int(max_ids),
                          _ptr(out["flags"]), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_trace rejected its arguments")
    if max_ids > 0:
        out["ids"], out["tau"] = ids, tau
    return out


def trace_alternatives(scene, ray_o, ray_d, params: Params = Params(), margins: Margins = Margins(),
                       max_alts: int = 256, n_threads: int = 0):
    """Admissible outcomes of each ray (see oracle_trace_alternatives in
    irgs_oracle.c): a candidate within a margin of a discontinuity in or out,
    runs of near-equal depths in any order, the T_min stop on either side.
    Returns feat [R,A,Fc], depth [R,A], opacity [R,A], n_hits [R,A] and
    count [R] (outcomes filled; -1 = too many to enumerate, where only the
    definition's own answer, outcome 0, is filled)."""
    lib = _load()
    means, quats, scales, opacity, feats = _surfel_arrays(scene)
    o, d = _f32(ray_o).reshape(-1, 3), _f32(ray_d).reshape(-1, 3)
    R, n, F = o.shape[0], means.shape[0], feats.shape[1]
    fc, A = params.feat_count, int(max_alts)
    out = {"feat": np.zeros((R, A, fc), np.float64), "depth": np.zeros((R, A), np.float64),
           "opacity": np.zeros((R, A), np.float64), "n_hits": np.zeros((R, A), np.int32),
           "count": np.zeros(R, np.int32)}
    p, m = params.c(), margins.c()
    rc = lib.oracle_trace_alternatives(_ptr(means), _ptr(quats), _ptr(scales), _ptr(opacity), _ptr(feats),
                                       n, F, _ptr(o), _ptr(d), R, C.byref(p), C.byref(m), A,
                                       _ptr(out["feat"]), _ptr(out["depth"]), _ptr(out["opacity"]),
                                       _ptr(out["n_hits"]), _ptr(out["count"]), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_trace_alternatives rejected its arguments")
    return out


def trace_grad(scene, ray_o, ray_d, g_feat, g_depth, g_opacity, params: Params = Params(),
               n_threads: int = 0):
    """Analytic FP64 gradient of sum(g_feat*feat + g_depth*depth + g_opacity*opacity)
    w.r.t. means, quats, scales, opacity, features (dict of float64 arrays)."""
    lib = _load()
    means, quats, scales, opacity, feats = _surfel_arrays(scene)
    o, d = _f32(ray_o).reshape(-1, 3), _f32(ray_d).reshape(-1, 3)
    R, n, F = o.shape[0], means.shape[0], feats.shape[1]
    gf = _f32(g_feat).reshape(R, params.feat_count)
    gd, go = _f32(g_depth).reshape(R), _f32(g_opacity).reshape(R)
    out = {"means": np.zeros((n, 3)), "quats": np.zeros((n, 4)), "scales": np.zeros((n, 2)),
           "opacity": np.zeros(n), "features": np.zeros((n, F))}
    p = params.c()
    rc = lib.oracle_trace_grad(_ptr(means), _ptr(quats), _ptr(scales), _ptr(opacity), _ptr(feats),
                               n, F, _ptr(o), _ptr(d), R, C.byref(p), _ptr(gf), _ptr(gd), _ptr(go),
                               _ptr(out["means"]), _ptr(out["quats"]), _ptr(out["scales"]),
                               _ptr(out["opacity"]), _ptr(out["features"]), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_trace_grad rejected its arguments")
    return out


MODE_SPLIT, MODE_UNIFORM = 0, 1


def _shade_inputs(scene, x, nrm, albedo, rough, wo, env):
    means, quats, scales, opacity, feats = _surfel_arrays(scene)
    x, nrm, albedo, wo = (_f32(a).reshape(-1, 3) for a in (x, nrm, albedo, wo))
    rough = _f32(rough).reshape(-1)
    env = _f32(env)
    return (means, quats, scales, opacity, feats), x, nrm, albedo, rough, wo, env


def shade(scene, x, nrm, albedo, rough, wo, env, n_diffuse: int, n_spec: int, seed: int,
          params: Params, margins: Margins | None = Margins(), n_threads: int = 0,
          point_ids=None, mode: int = MODE_SPLIT):
    """Monte Carlo rendering equation per point (Eq. 13-15). Returns a dict
    with rgb [P,3], vis [P], ind [P,3] and flags [P]. `point_ids` gives the
    point number that keys each point's random stream (default 0..P-1).
    mode MODE_SPLIT: n_diffuse cosine + n_spec GGX samples per point;
    MODE_UNIFORM: n_diffuse stratified uniform hemisphere samples (Eq. 15)."""
    lib = _load()
    (means, quats, scales, opacity, feats), x, nrm, albedo, rough, wo, env = _shade_inputs(
        scene, x, nrm, albedo, rough, wo, env)
    H, W = env.shape[0], env.shape[1]
    Pn, n, F = x.shape[0], means.shape[0], feats.shape[1]
    out = {"rgb": np.zeros((Pn, 3)), "vis": np.zeros(Pn), "ind": np.zeros((Pn, 3)),
           "flags": np.zeros(Pn, np.uint32)}
    p = params.c()
    m = margins.c() if margins is not None else None
    pid = None if point_ids is None else np.ascontiguousarray(point_ids, np.int64).reshape(Pn)
    rc = lib.oracle_shade(_ptr(means), _ptr(quats), _ptr(scales), _ptr(opacity), _ptr(feats), n, F,
                          _ptr(x), _ptr(nrm), _ptr(albedo), _ptr(rough), _ptr(wo), Pn, _ptr(env),
                          H, W, int(n_diffuse), int(n_spec), int(mode), C.c_uint64(seed & (2**64 - 1)),
                          _ptr(pid), C.byref(p), C.byref(m) if m is not None else None,
                          _ptr(out["rgb"]), _ptr(out["vis"]), _ptr(out["ind"]), _ptr(out["flags"]),
                          int(n_threads))
    if rc != 0:
        raise ValueError("oracle_shade rejected its arguments")
    return out


def shade_bounds(scene, x, nrm, albedo, rough, wo, env, n_diffuse: int, n_spec: int, seed: int,
                 params: Params, margins: Margins = Margins(), max_alts: int = 256, n_threads: int = 0,
                 point_ids=None, mode: int = MODE_SPLIT):
    """Admissible range of each point's shading estimate (oracle_shade_bounds
    in irgs_oracle.c): every sample's trace is one of its admissible outcomes
    (trace_alternatives). Returns lo [P,3], hi [P,3] and unresolved [P]
    (samples whose outcomes were too many to list)."""
    lib = _load()
    (means, quats, scales, opacity, feats), x, nrm, albedo, rough, wo, env = _shade_inputs(
        scene, x, nrm, albedo, rough, wo, env)
    Pn, n, F = x.shape[0], means.shape[0], feats.shape[1]
    out = {"lo": np.zeros((Pn, 3)), "hi": np.zeros((Pn, 3)), "unresolved": np.zeros(Pn, np.int32)}
    p, m = params.c(), margins.c()
    pid = None if point_ids is None else np.ascontiguousarray(point_ids, np.int64).reshape(Pn)
    rc = lib.oracle_shade_bounds(_ptr(means), _ptr(quats), _ptr(scales), _ptr(opacity), _ptr(feats), n, F,
                                 _ptr(x), _ptr(nrm), _ptr(albedo), _ptr(rough), _ptr(wo), Pn, _ptr(env),
                                 env.shape[0], env.shape[1], int(n_diffuse), int(n_spec), int(mode),
                                 C.c_uint64(seed & (2**64 - 1)), _ptr(pid), C.byref(p), C.byref(m), int(max_alts),
                                 _ptr(out["lo"]), _ptr(out["hi"]), _ptr(out["unresolved"]), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_shade_bounds rejected its arguments")
    return out


def shade_grad(scene, x, nrm, albedo, rough, wo, env, n_diffuse: int, n_spec: int, seed: int,
               params: Params, g_rgb, n_threads: int = 0, point_ids=None, mode: int = MODE_SPLIT,
               want_env: bool = True):
    """Gradient of sum(g_rgb * rgb) with the sample directions held fixed:
    dict of float64 arrays albedo [P,3], rough [P], env [H,W,3] and the
    surfel gradients means/quats/scales/opacity/features."""
    lib = _load()
    (means, quats, scales, opacity, feats), x, nrm, albedo, rough, wo, env = _shade_inputs(
        scene, x, nrm, albedo, rough, wo, env)
    H, W = env.shape[0], env.shape[1]
    Pn, n, F = x.shape[0], means.shape[0], feats.shape[1]
    g = _f32(g_rgb).reshape(Pn, 3)
    out = {"albedo": np.zeros((Pn, 3)), "rough": np.zeros(Pn),
           "env": np.zeros((H, W, 3)) if want_env else None,
           "means": np.zeros((n, 3)), "quats": np.zeros((n, 4)), "scales": np.zeros((n, 2)),
           "opacity": np.zeros(n), "features": np.zeros((n, F))}
    p = params.c()
    pid = None if point_ids is None else np.ascontiguousarray(point_ids, np.int64).reshape(Pn)
    rc = lib.oracle_shade_grad(_ptr(means), _ptr(quats), _ptr(scales), _ptr(opacity), _ptr(feats), n, F,
                               _ptr(x), _ptr(nrm), _ptr(albedo), _ptr(rough), _ptr(wo), Pn, _ptr(env),
                               H, W, int(n_diffuse), int(n_spec), int(mode), C.c_uint64(seed & (2**64 - 1)),
                               _ptr(pid), C.byref(p), _ptr(g), _ptr(out["albedo"]), _ptr(out["rough"]),
                               _ptr(out["env"]), _ptr(out["means"]), _ptr(out["quats"]), _ptr(out["scales"]),
                               _ptr(out["opacity"]), _ptr(out["features"]), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_shade_grad rejected its arguments")
    return out


def splitmix64(seed: int, i: int) -> int:
    """Output number i (0-based) of the SplitMix64 stream seeded with `seed`."""
    return int(_load().oracle_splitmix64(C.c_uint64(seed & (2**64 - 1)), C.c_uint64(i)))


def env_lookup(env, dirs):
    """Bilinear equirectangular lookup of directions [M,3] -> [M,3]."""
    lib = _load()
    env = _f32(env)
    dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    out = np.zeros_like(dirs)
    for i in range(dirs.shape[0]):
        lib.oracle_env_lookup(_ptr(env), env.shape[0], env.shape[1],
                              dirs[i].ctypes.data_as(C.c_void_p), out[i].ctypes.data_as(C.c_void_p))
    return out


def sample_dirs(nrm, wo, rough, n_diffuse: int, n_spec: int, seed: int, mode: int = 0):
    """Incident directions [P,S,3] and validity [P,S] of the shading samples."""
    lib = _load()
    nrm, wo = _f32(nrm).reshape(-1, 3), _f32(wo).reshape(-1, 3)
    rough = _f32(rough).reshape(-1)
    Pn, S = nrm.shape[0], n_diffuse + n_spec
    dirs = np.zeros((Pn, S, 3))
    valid = np.zeros((Pn, S), np.int32)
    lib.oracle_sample_dirs(_ptr(nrm), _ptr(wo), _ptr(rough), Pn, n_diffuse, n_spec, int(mode),
                           C.c_uint64(seed & (2**64 - 1)), _ptr(dirs), _ptr(valid))
    return dirs, valid.astype(bool)


# Sizes of the relighting maps (supplementary "Relighting details").
RL_IRR = (32, 64)
RL_LEVELS = 6
RL_PREF = (64, 128)
RL_LUT_N = 32


def relight_maps(env, n_threads: int = 0):
    """Pre-integrated maps of an environment [H,W,3]: irr [32,64,3] (diffuse
    irradiance), pref [5,64,128,3] (split-sum prefiltered radiance at
    roughness 0.2..1.0; level 0 is the environment), lut [32,32,2] (split-sum
    BRDF factors A, B over (n.v, roughness) cell centres), row_cdf [H+1] and
    col_cdf [H,W+1] (importance-sampling tables)."""
    env = _f32(env)
    H, W = env.shape[0], env.shape[1]
    out = {"irr": np.zeros(RL_IRR + (3,)), "pref": np.zeros((RL_LEVELS - 1,) + RL_PREF + (3,)),
           "lut": np.zeros((RL_LUT_N, RL_LUT_N, 2)), "row_cdf": np.zeros(H + 1), "col_cdf": np.zeros((H, W + 1))}
    rc = _load().oracle_relight_maps(_ptr(env), H, W, int(n_threads), _ptr(out["irr"]), _ptr(out["pref"]),
                                     _ptr(out["lut"]), _ptr(out["row_cdf"]), _ptr(out["col_cdf"]))
    if rc != 0:
        raise ValueError("oracle_relight_maps rejected its arguments")
    return out


def env_samples(env, P: int, S: int, seed: int):
    """Environment importance samples: directions [P,S,3] and pdf [P,S]."""
    env = _f32(env)
    dirs = np.zeros((P, S, 3))
    pdf = np.zeros((P, S))
    _load().oracle_env_samples(_ptr(env), env.shape[0], env.shape[1], P, S, C.c_uint64(seed & (2**64 - 1)),
                               _ptr(dirs), _ptr(pdf))
    return dirs, pdf


def relight(scene, x, nrm, albedo, rough, wo, env, n_samples: int, seed: int, params: Params,
            margins: Margins | None = Margins(), n_threads: int = 0, point_ids=None):
    """Relighting estimate per point under environment `env` (supplementary
    "Relighting details"): params.feat_offset / feat_count = 7 select the
    traced [albedo (3), roughness, normal (3)] channels. Returns rgb [P,3],
    vis [P], ind [P,3] and flags [P]."""
    lib = _load()
    (means, quats, scales, opacity, feats), x, nrm, albedo, rough, wo, env = _shade_inputs(
        scene, x, nrm, albedo, rough, wo, env)
    H, W = env.shape[0], env.shape[1]
    Pn, n, F = x.shape[0], means.shape[0], feats.shape[1]
    out = {"rgb": np.zeros((Pn, 3)), "vis": np.zeros(Pn), "ind": np.zeros((Pn, 3)),
           "flags": np.zeros(Pn, np.uint32)}
    p = params.c()
    m = margins.c() if margins is not None else None
    pid = None if point_ids is None else np.ascontiguousarray(point_ids, np.int64).reshape(Pn)
    rc = lib.oracle_relight(_ptr(means), _ptr(quats), _ptr(scales), _ptr(opacity), _ptr(feats), n, F,
                            _ptr(x), _ptr(nrm), _ptr(albedo), _ptr(rough), _ptr(wo), Pn, _ptr(env), H, W,
                            int(n_samples), C.c_uint64(seed & (2**64 - 1)), _ptr(pid), C.byref(p),
                            C.byref(m) if m is not None else None, _ptr(out["rgb"]), _ptr(out["vis"]),
                            _ptr(out["ind"]), _ptr(out["flags"]), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_relight rejected its arguments")
    return out


F_BRANCH = 128   # rasteriser: the 3D and screen-space terms of rho^2 nearly tie


class Camera(C.Structure):
    """Pinhole camera: pixel (px, py) looks along normalise(forward + x right
    + y up), x = ((px + 0.5)/width 2 - 1) tan_half_fov width/height,
    y = (1 - (py + 0.5)/height 2) tan_half_fov."""
    _fields_ = [("origin", C.c_float * 3), ("forward", C.c_float * 3), ("right", C.c_float * 3),
                ("up", C.c_float * 3), ("tan_half_fov", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


def camera(origin, forward, right, up, tan_half_fov, width, height) -> Camera:
    c = Camera()
    c.origin[:] = [float(v) for v in origin]
    c.forward[:] = [float(v) for v in forward]
    c.right[:] = [float(v) for v in right]
    c.up[:] = [float(v) for v in up]
    c.tan_half_fov = float(tan_half_fov)
    c.width, c.height = int(width), int(height)
    return c


def rasterize(scene, cam: Camera, params: Params = Params(), margins: Margins | None = Margins(),
              n_threads: int = 0):
    """2D Gaussian rasterisation of a width x height image (row-major): the
    surfels with centre view depth > params.t_min blended in centre-depth
    order with the 2DGS low-pass filter. Returns feat [P,Fc], depth [P],
    opacity [P], n_hits [P], flags [P]."""
    lib = _load()
    means, quats, scales, opacity, feats = _surfel_arrays(scene)
    n, F = means.shape[0], feats.shape[1]
    Pn = cam.width * cam.height
    out = {"feat": np.zeros((Pn, params.feat_count)), "depth": np.zeros(Pn), "opacity": np.zeros(Pn),
           "n_hits": np.zeros(Pn, np.int32), "flags": np.zeros(Pn, np.uint32)}
    p = params.c()
    m = margins.c() if margins is not None else None
    rc = lib.oracle_rasterize(_ptr(means), _ptr(quats), _ptr(scales), _ptr(opacity), _ptr(feats), n, F,
                              C.byref(cam), C.byref(p), C.byref(m) if m is not None else None, _ptr(out["feat"]),
                              _ptr(out["depth"]), _ptr(out["opacity"]), _ptr(out["n_hits"]), _ptr(out["flags"]),
                              int(n_threads))
    if rc != 0:
        raise ValueError("oracle_rasterize rejected its arguments")
    return out


def relight_bounds(scene, x, nrm, albedo, rough, wo, env, n_samples: int, seed: int, params: Params,
                   margins: Margins = Margins(), max_alts: int = 256, n_threads: int = 0, point_ids=None):
    """Admissible range of each point's relighting estimate
    (oracle_relight_bounds in irgs_oracle.c). Returns lo [P,3], hi [P,3] and
    unresolved [P]."""
    lib = _load()
    (means, quats, scales, opacity, feats), x, nrm, albedo, rough, wo, env = _shade_inputs(
        scene, x, nrm, albedo, rough, wo, env)
    Pn, n, F = x.shape[0], means.shape[0], feats.shape[1]
    out = {"lo": np.zeros((Pn, 3)), "hi": np.zeros((Pn, 3)), "unresolved": np.zeros(Pn, np.int32)}
    p, m = params.c(), margins.c()
    pid = None if point_ids is None else np.ascontiguousarray(point_ids, np.int64).reshape(Pn)
    rc = lib.oracle_relight_bounds(_ptr(means), _ptr(quats), _ptr(scales), _ptr(opacity), _ptr(feats), n, F,
                                   _ptr(x), _ptr(nrm), _ptr(albedo), _ptr(rough), _ptr(wo), Pn, _ptr(env),
                                   env.shape[0], env.shape[1], int(n_samples), C.c_uint64(seed & (2**64 - 1)),
                                   _ptr(pid), C.byref(p), C.byref(m), int(max_alts), _ptr(out["lo"]),
                                   _ptr(out["hi"]), _ptr(out["unresolved"]), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_relight_bounds rejected its arguments")
    return out
