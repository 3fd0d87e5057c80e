"""Pins of the oracle's 2D Gaussian rasterisation (centre-depth order, 2DGS
low-pass filter): closed forms for one surfel, the filter for a sub-pixel
surfel, the order rule, the near plane, and agreement with the brute-force
tracer where the two definitions coincide (fronto-parallel surfels much
larger than a pixel)."""
import math

import numpy as np

import oracle
from tests.helpers import scene

P3 = oracle.Params(feat_count=3)


def cam_z(width=24, height=16, fov=40.0, z=5.0):
    """Camera at (0,0,z) looking down -z: right = +x, up = +y."""
    return oracle.camera((0, 0, z), (0, 0, -1), (1, 0, 0), (0, 1, 0), math.tan(math.radians(fov) / 2), width, height)


def pixel_ray(c, px, py):
    W, H = c.width, c.height
    sx = (px + 0.5) / W * 2 - 1
    sy = 1 - (py + 0.5) / H * 2
    f, r, u = (np.array(v[:], np.float64) for v in (c.forward, c.right, c.up))
    d = f + sx * c.tan_half_fov * (W / H) * r + sy * c.tan_half_fov * u
    return d / np.linalg.norm(d)


def one(mean, scale, o, quat=(1, 0, 0, 0), f=(1.0, 0.5, 0.25)):
    return scene(np.array([mean], np.float32), np.array([quat], np.float32), np.array([scale], np.float32),
                 np.array([o], np.float32), np.array([f], np.float32))


def test_single_facing_surfel_closed_form():
    c = cam_z()
    sc = one((0.3, -0.2, 0.0), (0.8, 0.5), 0.7)
    out = oracle.rasterize(sc, c, P3, margins=None)
    for px, py in [(0, 0), (12, 8), (15, 5), (20, 13), (7, 10)]:
        d = pixel_ray(c, px, py)
        t = 5.0 / -d[2]                                   # plane z = 0
        p = np.array([0, 0, 5.0]) + t * d
        mx, my, su, sv, o = (float(np.float32(v)) for v in (0.3, -0.2, 0.8, 0.5, 0.7))
        rho2 = ((p[0] - mx) / su) ** 2 + ((p[1] - my) / sv) ** 2
        a = o * math.exp(-rho2 / 2) if rho2 <= 9 else 0.0
        a = a if a >= 1 / 255 else 0.0
        i = py * c.width + px
        assert abs(out["opacity"][i] - a) < 1e-12, (px, py)
        assert abs(out["depth"][i] - a * t) < 1e-12
        np.testing.assert_allclose(out["feat"][i], a * np.array([1.0, 0.5, 0.25]), atol=1e-12)


def test_subpixel_surfel_follows_the_screen_space_filter():
    c = cam_z(width=32, height=32, fov=30.0)
    mean = np.array([0.11, 0.07, 0.0], np.float32).astype(np.float64)
    sc = one(mean, (1e-5, 1e-5), 0.9)
    out = oracle.rasterize(sc, c, P3, margins=None)
    # projected centre in pixel coordinates (pixel centres at integers)
    tf = c.tan_half_fov
    pxc = (mean[0] / 5.0 / tf + 1) * 0.5 * 32 - 0.5
    pyc = (1 - mean[1] / 5.0 / tf) * 0.5 * 32 - 0.5
    for px in range(32):
        for py in range(32):
            r2 = ((px - pxc) ** 2 + (py - pyc) ** 2) / 0.5
            a = float(np.float32(0.9)) * math.exp(-r2 / 2) if r2 <= 9 else 0.0
            a = a if a >= 1 / 255 else 0.0
            assert abs(out["opacity"][py * 32 + px] - a) < 1e-9, (px, py)
    assert (out["n_hits"] > 0).sum() >= 4


def test_blend_order_is_centre_depth_not_intersection_depth():
    """A tilted surfel B whose centre lies behind a fronto-parallel one A but
    whose plane the centre pixel's ray crosses first: the tracer blends B
    first, the rasteriser A (the nearer centre)."""
    c = cam_z(width=8, height=8, fov=10.0)
    qa, qb = [1, 0, 0, 0], [math.cos(0.6), -math.sin(0.6), 0, 0]     # B: ~69 deg about x
    ma, mb = [0, 0, 0.0], [0, 0.3, -0.2]

    def mk(idx):
        m = np.array([ma, mb], np.float32)[idx]
        q = np.array([qa, qb], np.float32)[idx]
        s_ = np.array([[0.5, 0.5], [2.0, 2.0]], np.float32)[idx]
        o = np.array([0.6, 0.8], np.float32)[idx]
        f = np.array([[1, 0, 0], [0, 1, 0]], np.float32)[idx]
        return scene(m, q, s_, o, f)
    i = 3 * 8 + 3
    d = pixel_ray(c, 3, 3)[None].astype(np.float32)
    ro = np.array([[0, 0, 5.0]], np.float32)
    ras = {k: oracle.rasterize(mk(idx), c, P3, margins=None) for k, idx in (("AB", [0, 1]), ("A", [0]), ("B", [1]))}
    tr = {k: oracle.trace(mk(idx), ro, d, P3, margins=None) for k, idx in (("AB", [0, 1]), ("A", [0]), ("B", [1]))}
    aA, aB = ras["A"]["opacity"][i], ras["B"]["opacity"][i]
    assert aA > 0.3 and aB > 0.3
    np.testing.assert_allclose(ras["AB"]["feat"][i], [aA, (1 - aA) * aB, 0], atol=1e-12)
    tA, tB = tr["A"]["opacity"][0], tr["B"]["opacity"][0]
    np.testing.assert_allclose(tr["AB"]["feat"][0], [(1 - tB) * tA, tB, 0], atol=1e-6)


def test_near_plane_and_surfels_behind_the_camera():
    c = cam_z()
    for z in (5.5, 4.95):                                           # behind, and closer than t_min = 0.1
        sc = one((0, 0, z), (1.0, 1.0), 0.9)
        out = oracle.rasterize(sc, c, oracle.Params(feat_count=3, t_min=0.1), margins=None)
        assert out["opacity"].max() == 0.0


def test_matches_the_tracer_for_large_fronto_parallel_surfels():
    rng = np.random.default_rng(7)
    m = 40
    means = np.c_[rng.uniform(-1, 1, m), rng.uniform(-1, 1, m), rng.uniform(-1.5, 1.5, m)].astype(np.float32)
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (m, 1))
    quats[:, 3] = rng.uniform(-0.3, 0.3, m)                        # in-plane rotation only
    scales = rng.uniform(0.3, 0.6, size=(m, 2)).astype(np.float32)
    sc = scene(means, quats, scales, rng.uniform(0.2, 0.9, m).astype(np.float32),
               rng.uniform(0, 1, size=(m, 3)).astype(np.float32))
    c = cam_z(width=40, height=30, fov=35.0, z=6.0)
    ras = oracle.rasterize(sc, c, P3)
    rays = np.array([pixel_ray(c, px, py) for py in range(30) for px in range(40)], np.float32)
    ro = np.tile(np.array([0, 0, 6.0], np.float32), (rays.shape[0], 1))
    tr = oracle.trace(sc, ro, rays, P3)
    ok = (ras["flags"] == 0) & (tr["flags"] == 0)
    assert ok.mean() > 0.9 and (ras["n_hits"][ok] > 2).mean() > 0.5
    np.testing.assert_allclose(ras["feat"][ok], tr["feat"][ok], atol=1e-6)
    np.testing.assert_allclose(ras["opacity"][ok], tr["opacity"][ok], atol=1e-6)
    np.testing.assert_allclose(ras["depth"][ok], tr["depth"][ok], atol=1e-5)
    np.testing.assert_array_equal(ras["n_hits"][ok], tr["n_hits"][ok])
