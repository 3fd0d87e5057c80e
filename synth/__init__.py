"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA tracer.

This module only *generates inputs*: surfel clouds, camera rays, G-buffers,
environment maps and upstream gradients, all as float32 NumPy arrays. It holds
none of the tracer's arithmetic (no ray/surfel intersection, no compositing, no
BRDF): the oracle and the CUDA path each implement that on their own. Both
sides consume exactly the same float32 arrays.

The shapes mirror the object-centric workloads of IRGS (2D Gaussian surfels
on object surfaces, Sec. 3.2; camera rays and Monte Carlo incident rays,
Eq. 8 and Eq. 14-15). The datasets of the paper (Synthetic4Relight, TensoIR,
Stanford-ORB) are not available; these scenes stand in for their shape.

Conventions
-----------
* quaternions are (w, x, y, z); rotation columns are (t_u, t_v, n);
* scales are (s_u, s_v) > 0, opacity in (0, 1), both already activated;
* ray directions are unit length in float64 and then rounded to float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Surfels", "tiny_scene", "object_scene", "object_scene_median_scale",
    "look_at_rays", "tiny_camera", "hemisphere_cameras", "camera_batch_rays",
    "gbuffer_points", "env_map", "upstream_grads", "random_rays_through_scene",
    "frame_to_quat", "tile_order",
]

# Scene geometry of the object-centric stand-in (sphere, torus, ground).
SPHERE_C = np.array([-1.1, 0.0, 1.0])
SPHERE_R = 1.0
TORUS_C = np.array([1.1, 0.0, 0.25])
TORUS_R, TORUS_r = 0.7, 0.25
GROUND_HALF = 2.5


@dataclass
class Surfels:
    """A cloud of 2D Gaussian surfels (float32, user order)."""
    means: np.ndarray      # [N, 3]
    quats: np.ndarray      # [N, 4] (w, x, y, z)
    scales: np.ndarray     # [N, 2]
    opacity: np.ndarray    # [N]
    features: np.ndarray   # [N, F]

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self):
        return self.means, self.quats, self.scales, self.opacity, self.features

    def subset(self, idx) -> "Surfels":
        idx = np.asarray(idx)
        return Surfels(*(np.ascontiguousarray(a[idx]) for a in self.arrays()))


def frame_to_quat(t_u: np.ndarray, t_v: np.ndarray, n: np.ndarray) -> np.ndarray:
    """Unit quaternion (w,x,y,z) of the rotation whose columns are (t_u,t_v,n).

    Uses SciPy's matrix-to-quaternion conversion (input generation only).
    """
    from scipy.spatial.transform import Rotation

    m = np.stack([t_u, t_v, n], axis=-1)           # columns
    xyzw = Rotation.from_matrix(m).as_quat()
    return np.concatenate([xyzw[:, 3:4], xyzw[:, :3]], axis=1)


def tiny_scene(seed: int = 1000, n: int = 1024, n_feat: int = 3) -> Surfels:
    """Tiny random cloud: centres U[-1,1]^3, uniform rotations, log-uniform
    scales in [0.02, 0.2], opacity U(0.05, 0.95), features U[0,1]."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(n, 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    scales = np.exp(rng.uniform(math.log(0.02), math.log(0.2), size=(n, 2)))
    opacity = rng.uniform(0.05, 0.95, size=n)
    feats = rng.uniform(0.0, 1.0, size=(n, n_feat))
    return Surfels(*(np.ascontiguousarray(a, dtype=np.float32)
                     for a in (means, q, scales, opacity, feats)))


def object_scene_median_scale(n: int) -> float:
    """Median surfel scale that keeps per-ray depth complexity constant:
    0.01 at 300k surfels, scaled by sqrt(300k / n)."""
    return 0.01 * math.sqrt(300_000.0 / float(n))


def _sample_torus(rng, m):
    # area element of the torus ~ (R + r cos v): rejection on v
    out_v = np.empty(0)
    while out_v.size < m:
        v = rng.uniform(0.0, 2 * math.pi, size=2 * m)
        keep = rng.uniform(0.0, 1.0, size=2 * m) < (TORUS_R + TORUS_r * np.cos(v)) / (TORUS_R + TORUS_r)
        out_v = np.concatenate([out_v, v[keep]])
    v = out_v[:m]
    u = rng.uniform(0.0, 2 * math.pi, size=m)
    cu, su, cv, sv = np.cos(u), np.sin(u), np.cos(v), np.sin(v)
    p = np.stack([(TORUS_R + TORUS_r * cv) * cu, (TORUS_R + TORUS_r * cv) * su, TORUS_r * sv], 1) + TORUS_C
    nrm = np.stack([cv * cu, cv * su, sv], 1)
    return p, nrm


def _surface_points(rng, n):
    """n points on (sphere, torus, ground square) allocated by area, with
    their analytic outward normals. Returns (p, normal, shape_id)."""
    a_s = 4 * math.pi * SPHERE_R ** 2
    a_t = 4 * math.pi ** 2 * TORUS_R * TORUS_r
    a_g = (2 * GROUND_HALF) ** 2
    tot = a_s + a_t + a_g
    n_s = int(round(n * a_s / tot))
    n_t = int(round(n * a_t / tot))
    n_g = n - n_s - n_t
    g = rng.normal(size=(n_s, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    p_s, n_s_ = SPHERE_C + SPHERE_R * g, g
    p_t, n_t_ = _sample_torus(rng, n_t)
    xy = rng.uniform(-GROUND_HALF, GROUND_HALF, size=(n_g, 2))
    p_g = np.concatenate([xy, np.zeros((n_g, 1))], 1)
    n_g_ = np.tile(np.array([0.0, 0.0, 1.0]), (n_g, 1))
    p = np.concatenate([p_s, p_t, p_g])
    nr = np.concatenate([n_s_, n_t_, n_g_])
    sid = np.concatenate([np.zeros(n_s, np.int32), np.ones(n_t, np.int32), np.full(n_g, 2, np.int32)])
    return p, nr, sid


def _tangent_frame(rng, nrm):
    """Random in-plane tangent t_u, t_v = n x t_u (right-handed frame)."""
    helper = np.where(np.abs(nrm[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    a = np.cross(helper, nrm)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = np.cross(nrm, a)
    ang = rng.uniform(0.0, 2 * math.pi, size=(nrm.shape[0], 1))
    t_u = np.cos(ang) * a + np.sin(ang) * b
    t_v = np.cross(nrm, t_u)
    return t_u, t_v


def object_scene(n: int = 300_000, seed: int = 1001, median_scale: float | None = None,
                 normal_jitter: float = 0.01, scale_sigma: float = 0.5) -> Surfels:
    """Object-centric scene: surfels tangent to a unit sphere, a torus and a
    ground square, normals jittered by N(0, jitter^2) per component, scales
    log-normal around `median_scale`, opacity Beta(5,1), 10 feature channels
    (radiance RGB, albedo RGB, roughness, normal xyz)."""
    rng = np.random.default_rng(seed)
    if median_scale is None:
        median_scale = object_scene_median_scale(n)
    p, nrm, _ = _surface_points(rng, n)
    nrm = nrm + rng.normal(scale=normal_jitter, size=nrm.shape)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    t_u, t_v = _tangent_frame(rng, nrm)
    q = frame_to_quat(t_u, t_v, nrm)
    scales = np.exp(rng.normal(math.log(median_scale), scale_sigma, size=(n, 2)))
    opacity = rng.beta(5.0, 1.0, size=n)
    opacity = np.clip(opacity, 1e-4, 1.0 - 1e-6)
    radiance = rng.uniform(0.0, 1.0, size=(n, 3))
    albedo = rng.uniform(0.05, 0.95, size=(n, 3))
    rough = rng.uniform(0.05, 1.0, size=(n, 1))
    feats = np.concatenate([radiance, albedo, rough, nrm], axis=1)
    return Surfels(*(np.ascontiguousarray(a, dtype=np.float32)
                     for a in (p, q, scales, opacity, feats)))


def tile_order(width: int, height: int, tile=(8, 4)) -> np.ndarray:
    """Pixel indices (row-major numbering) listed tile by tile: tiles of
    tile[0] x tile[1] pixels in row-major tile order, row-major inside a tile.
    Edge tiles are clipped when the image is not a multiple of the tile."""
    tw, th = tile
    ys, xs = np.mgrid[0:height, 0:width]
    key = ((ys // th) * ((width + tw - 1) // tw) + xs // tw) * (tw * th) + (ys % th) * tw + xs % tw
    return np.argsort(key.reshape(-1), kind="stable")


def look_at_rays(pos, target=(0.0, 0.0, 0.0), width: int = 64, height: int = 64,
                 fov_deg: float = 60.0, tile=None):
    """Pinhole camera rays through pixel centres (row-major, top row first,
    or tile by tile if `tile` = (tw, th) is given).

    z-up; if the view direction is within ~8 degrees of z, x is used as up.
    Returns float32 (origins [H*W,3], unit directions [H*W,3])."""
    pos = np.asarray(pos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) <= 0.99 else np.array([1.0, 0.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    up2 = np.cross(right, fwd)
    th = math.tan(math.radians(fov_deg) * 0.5)
    aspect = width / height
    xs = ((np.arange(width) + 0.5) / width * 2.0 - 1.0) * th * aspect
    ys = (1.0 - (np.arange(height) + 0.5) / height * 2.0) * th
    X, Y = np.meshgrid(xs, ys)
    d = fwd[None, :] + X.reshape(-1, 1) * right[None, :] + Y.reshape(-1, 1) * up2[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    if tile is not None:
        d = d[tile_order(width, height, tile)]
    o = np.broadcast_to(pos, d.shape)
    return np.ascontiguousarray(o, dtype=np.float32), np.ascontiguousarray(d, dtype=np.float32)


def tiny_camera(seed: int = 1000, radius: float = 3.0):
    """One camera position uniform on a sphere of the given radius."""
    rng = np.random.default_rng(seed + 7)
    v = rng.normal(size=3)
    return radius * v / np.linalg.norm(v)


def hemisphere_cameras(n: int = 100, seed: int = 1001, radius: float = 4.0,
                       min_elev_deg: float = 5.0) -> np.ndarray:
    """n camera positions uniform on the spherical cap above `min_elev_deg`."""
    rng = np.random.default_rng(seed + 11)
    z = rng.uniform(math.sin(math.radians(min_elev_deg)), 1.0, size=n)
    phi = rng.uniform(0.0, 2 * math.pi, size=n)
    r = np.sqrt(1.0 - z * z)
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)


def camera_batch_rays(cams: np.ndarray, width: int = 800, height: int = 800,
                      fov_deg: float = 60.0, out_o=None, out_d=None, tile=None):
    """Rays of several cameras, concatenated camera-major (float32); pixels
    row-major or tile by tile (see look_at_rays)."""
    m = width * height
    n = cams.shape[0] * m
    if out_o is None:
        out_o = np.empty((n, 3), np.float32)
    if out_d is None:
        out_d = np.empty((n, 3), np.float32)
    for i, c in enumerate(cams):
        o, d = look_at_rays(c, (0.0, 0.0, 0.0), width, height, fov_deg, tile)
        out_o[i * m:(i + 1) * m] = o
        out_d[i * m:(i + 1) * m] = d
    return out_o, out_d


def random_rays_through_scene(n: int, seed: int, box: float = 1.0, radius: float = 3.0):
    """Rays from random points on a sphere aimed at random points of a box:
    an incoherent ray set for tests."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    o = radius * v / np.linalg.norm(v, axis=1, keepdims=True)
    tgt = rng.uniform(-box, box, size=(n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.ascontiguousarray(o, np.float32), np.ascontiguousarray(d, np.float32)


def gbuffer_points(n_points: int = 640_000, seed: int = 1002, n_cams: int = 100):
    """Surface points of the object scene seen from the hemisphere cameras.

    Points lie on the analytic surfaces (area-weighted); each is paired with
    a random camera it faces, which gives the outgoing direction w_o.
    Albedo U[0.05,0.95]^3, roughness U[0.05,1]. Returns float32 arrays
    x[P,3], n[P,3], albedo[P,3], rough[P], wo[P,3]."""
    rng = np.random.default_rng(seed)
    cams = hemisphere_cameras(n_cams, seed=1001)
    xs, ns, wos = [], [], []
    have = 0
    while have < n_points:
        m = int((n_points - have) * 1.3) + 64
        p, nr, _ = _surface_points(rng, m)
        ci = rng.integers(0, n_cams, size=m)
        wo = cams[ci] - p
        wo /= np.linalg.norm(wo, axis=1, keepdims=True)
        ok = np.einsum("ij,ij->i", wo, nr) > 0.05
        xs.append(p[ok]); ns.append(nr[ok]); wos.append(wo[ok])
        have += int(ok.sum())
    x = np.concatenate(xs)[:n_points]
    nr = np.concatenate(ns)[:n_points]
    wo = np.concatenate(wos)[:n_points]
    albedo = rng.uniform(0.05, 0.95, size=(n_points, 3))
    rough = rng.uniform(0.05, 1.0, size=n_points)
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return f(x), f(nr), f(albedo), f(rough), f(wo)


def env_map(seed: int = 1003, height: int = 256, width: int = 512, n_lobes: int = 3,
            lobe_sigma_deg: float = 3.0, lobe_peak: float = 50.0) -> np.ndarray:
    """Equirectangular HDR map [H, W, 3] float32 (row = polar angle from +z,
    column = azimuth from -pi). Texels: LogNormal(0,1) x tint U[0.8,1.2]^3,
    plus `n_lobes` white Gaussian lobes (angular sigma, peak) at random
    upper-hemisphere directions."""
    rng = np.random.default_rng(seed)
    inten = rng.lognormal(0.0, 1.0, size=(height, width, 1))
    tint = rng.uniform(0.8, 1.2, size=(height, width, 3))
    env = inten * tint
    th = (np.arange(height) + 0.5) / height * math.pi
    ph = (np.arange(width) + 0.5) / width * 2 * math.pi - math.pi
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    dirs = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1)
    sig = math.radians(lobe_sigma_deg)
    for _ in range(n_lobes):
        z = rng.uniform(0.1, 1.0)
        phi = rng.uniform(0, 2 * math.pi)
        r = math.sqrt(1 - z * z)
        c = np.array([r * math.cos(phi), r * math.sin(phi), z])
        ang = np.arccos(np.clip(dirs @ c, -1.0, 1.0))
        env += lobe_peak * np.exp(-0.5 * (ang / sig) ** 2)[..., None]
    return np.ascontiguousarray(env, dtype=np.float32)


def upstream_grads(n_rays: int, n_feat: int, seed: int = 1004):
    """Random upstream gradients N(0,1): (g_feat [R,F], g_depth [R], g_opacity [R])."""
    rng = np.random.default_rng(seed)
    return (np.ascontiguousarray(rng.normal(size=(n_rays, n_feat)), np.float32),
            np.ascontiguousarray(rng.normal(size=n_rays), np.float32),
            np.ascontiguousarray(rng.normal(size=n_rays), np.float32))
