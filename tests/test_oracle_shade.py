"""Pins of the oracle's Monte Carlo rendering equation (Eq. 3, 4, 13-15):
a published RNG test vector, furnace tests with closed-form answers, an
adaptive-quadrature value of the specular lobe, sampler moments and the
environment lookup at texel centres."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import Params
from tests.helpers import scene

HERE = os.path.dirname(os.path.abspath(__file__))
PS = Params(alpha_min=1 / 255, alpha_max=0.99, T_min=1e-4, t_min=1e-3, feat_offset=0, feat_count=3)


def empty_scene():
    z = np.zeros((0, 3), np.float32)
    return scene(z, np.zeros((0, 4)), np.zeros((0, 2)), np.zeros(0), np.zeros((0, 3)))


def test_splitmix64_published_vector():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    for idx, hexv in rows:
        assert oracle.splitmix64(0, int(idx)) == int(hexv, 16)


def test_env_lookup_texel_centres_wrap_and_clamp():
    H, W = 8, 16
    rng = np.random.default_rng(0)
    env = rng.uniform(0, 10, size=(H, W, 3)).astype(np.float32)
    e64 = env.astype(np.float64)
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    th = (ii.reshape(-1) + 0.5) / H * math.pi
    ph = (jj.reshape(-1) + 0.5) / W * 2 * math.pi - math.pi
    dirs = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    got = oracle.env_lookup(env, dirs)
    np.testing.assert_allclose(got, env.reshape(-1, 3), rtol=1e-9, atol=1e-9)
    # azimuth +-pi sits halfway between the last and the first column
    t = (3 + 0.5) / H * math.pi
    d = np.array([[-math.sin(t), 0.0, math.cos(t)]])
    np.testing.assert_allclose(oracle.env_lookup(env, d)[0], 0.5 * (e64[3, 0] + e64[3, W - 1]), rtol=1e-9)
    # the pole clamps to the first row (horizontal interpolation only)
    up = oracle.env_lookup(env, np.array([[0.0, 0.0, 1.0]]))[0]
    x = (0.0 + math.pi) / (2 * math.pi) * W - 0.5
    j0 = int(math.floor(x))
    fx = x - j0
    np.testing.assert_allclose(up, (1 - fx) * e64[0, j0] + fx * e64[0, (j0 + 1) % W], rtol=1e-9)


def _points(P, n=(0.0, 0.0, 1.0), wo=(0.3, -0.2, 0.9), a=(0.6, 0.3, 0.15), r=0.5):
    n = np.tile(np.asarray(n, np.float32), (P, 1))
    wo = np.asarray(wo, np.float64)
    wo = np.tile((wo / np.linalg.norm(wo)).astype(np.float32), (P, 1))
    x = np.zeros((P, 3), np.float32)
    return x, n, np.tile(np.asarray(a, np.float32), (P, 1)), np.full(P, r, np.float32), wo


def test_diffuse_furnace_is_exact():
    # empty scene, constant environment L: every cosine sample returns a*L
    L = np.array([1.7, 0.4, 2.5], np.float32)
    env = np.tile(L, (16, 32, 1))
    x, n, a, r, wo = _points(7)
    out = oracle.shade(empty_scene(), x, n, a, r, wo, env, 24, 0, 1234, PS)
    np.testing.assert_allclose(out["rgb"], a.astype(np.float64) * L, rtol=1e-12)
    np.testing.assert_allclose(out["vis"], 1.0)
    np.testing.assert_allclose(out["ind"], 0.0)


def _spec_albedo_quadrature(rough, cos_o, F0=0.04):
    """Adaptive quadrature of int f_s (n.w_i) dw_i over the hemisphere."""
    ag = rough * rough
    a2 = ag * ag
    k = ag / 2
    wo = np.array([math.sqrt(1 - cos_o ** 2), 0.0, cos_o])

    def f(th, ph):
        wi = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        h = wi + wo
        h /= np.linalg.norm(h)
        nh, oh, ni = h[2], wo @ h, wi[2]
        D = a2 / (math.pi * (nh * nh * (a2 - 1) + 1) ** 2)
        F = F0 + (1 - F0) * (1 - oh) ** 5
        G = (ni / (ni * (1 - k) + k)) * (cos_o / (cos_o * (1 - k) + k))
        return D * F * G / (4 * ni * cos_o) * ni * math.sin(th)

    val, _ = integrate.dblquad(lambda th, ph: f(th, ph), 0, 2 * math.pi, 0, math.pi / 2,
                               epsabs=1e-7, epsrel=1e-6)
    return val


@pytest.mark.parametrize("rough,theta_o_deg", [(0.5, 30.0), (0.9, 60.0), (0.7, 10.0)])
def test_specular_furnace_converges_to_quadrature(rough, theta_o_deg):
    co = math.cos(math.radians(theta_o_deg))
    wo = (math.sqrt(1 - co * co), 0.0, co)
    P = 48
    x, n, a, r, wo_a = _points(P, wo=wo, a=(0.0, 0.0, 0.0), r=rough)
    env = np.ones((16, 32, 3), np.float32)
    out = oracle.shade(empty_scene(), x, n, a, r, wo_a, env, 0, 2048, 99, PS)
    est = out["rgb"][:, 0]
    mean, sem = est.mean(), est.std(ddof=1) / math.sqrt(P)
    ref = _spec_albedo_quadrature(float(r[0]), float(np.float64(wo_a[0]) @ np.array([0, 0, 1.0])))
    assert abs(mean - ref) < 4.5 * sem + 1e-6, (mean, ref, sem)
    # channels are equal (scalar F0, white light)
    np.testing.assert_allclose(out["rgb"][:, 1], est)


def test_cosine_sampler_moments():
    nrm = np.array([[0.3, -0.5, 0.8]], np.float32)
    wo = nrm.copy()
    dirs, valid = oracle.sample_dirs(nrm, wo, np.array([0.5], np.float32), 20000, 0, 5)
    nn = nrm[0].astype(np.float64) / np.linalg.norm(nrm[0])
    c = dirs[0] @ nn
    assert valid.all() and np.all(c > 0)
    np.testing.assert_allclose(np.linalg.norm(dirs[0], axis=1), 1.0, atol=1e-12)
    # E[cos] = 2/3, E[cos^2] = 1/2 under the cosine-weighted density
    assert abs(c.mean() - 2 / 3) < 4 * c.std() / math.sqrt(c.size)
    assert abs((c * c).mean() - 0.5) < 4 * (c * c).std() / math.sqrt(c.size)
    # azimuth uniform: the mean tangent component vanishes
    t = dirs[0] - np.outer(c, nn)
    assert np.all(np.abs(t.mean(0)) < 4 * t.std(0) / math.sqrt(c.size))


def test_ggx_samples_reflect_about_half_vector():
    nrm = np.array([[0.0, 0.0, 1.0]], np.float32)
    wo = np.array([[0.5, 0.0, math.sqrt(0.75)]], np.float32)
    dirs, valid = oracle.sample_dirs(nrm, wo, np.array([0.3], np.float32), 0, 4000, 17)
    w = dirs[0][valid[0]]
    assert np.all(w[:, 2] > 0)
    # low roughness: reflected directions concentrate around the mirror direction
    mirror = np.array([-0.5, 0.0, math.sqrt(0.75)])
    assert np.median(w @ mirror) > 0.95


def test_opaque_canopy_light_decomposition():
    # one huge disk 1 unit above the point: each traced ray returns
    # L_ind = alpha f and V = 1 - alpha, so L_i = V L + (1 - V) f exactly
    f = np.array([0.2, 0.9, 0.4])
    sc = scene([0, 0, 1.0], [1, 0, 0, 0], [100.0, 100.0], [0.5], f)
    L = np.array([2.0, 1.0, 0.5], np.float32)
    env = np.tile(L, (16, 32, 1))
    x, n, a, r, wo = _points(5)
    out = oracle.shade(sc, x, n, a, r, wo, env, 32, 0, 7, PS)
    vis = out["vis"]
    assert np.all(vis >= 0.5 - 1e-12) and np.all(vis < 0.51)
    expect = a.astype(np.float64) * (vis[:, None] * L + (1 - vis[:, None]) * sc.features[0].astype(np.float64))
    np.testing.assert_allclose(out["rgb"], expect, rtol=1e-12)
    np.testing.assert_allclose(out["ind"], (1 - vis[:, None]) * sc.features[0].astype(np.float64), rtol=1e-12)


def test_backfacing_normal_is_flipped():
    x, n, a, r, wo = _points(4)
    env = np.random.default_rng(3).uniform(0, 5, size=(16, 32, 3)).astype(np.float32)
    o1 = oracle.shade(empty_scene(), x, n, a, r, wo, env, 8, 8, 5, PS)
    o2 = oracle.shade(empty_scene(), x, -n, a, r, wo, env, 8, 8, 5, PS)
    np.testing.assert_allclose(o1["rgb"], o2["rgb"], rtol=1e-12)


def test_secondary_ray_starts_after_t_min():
    # a surfel through the shading point itself is skipped (tau ~ 0 < t_min)
    sc = scene([0, 0, 0], [1, 0, 0, 0], [1.0, 1.0], [0.9], [1, 1, 1])
    env = np.ones((16, 32, 3), np.float32)
    x, n, a, r, wo = _points(3)
    out = oracle.shade(sc, x, n, a, r, wo, env, 16, 0, 3, PS)
    np.testing.assert_allclose(out["vis"], 1.0)
