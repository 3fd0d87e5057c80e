"""Pins of the oracle's relighting query (supplementary "Relighting details",
Eq. 18): the pre-integrated maps against quadrature and closed forms, the
environment sampler against its texel probabilities, and the estimator in
cases whose answer is known independently of the oracle's own tables.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from tests.helpers import scene

PR = oracle.Params(alpha_min=1 / 255, alpha_max=0.99, T_min=1e-4, t_min=1e-3, feat_offset=0, feat_count=7)


def sph(th, ph):
    return np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])


def texel_centres(h, w):
    th = (np.arange(h) + 0.5) * math.pi / h
    ph = (np.arange(w) + 0.5) * 2 * math.pi / w - math.pi
    T, P = np.meshgrid(th, ph, indexing="ij")
    return np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1)


def sphere_quad(f, eps=1e-7):
    """Integral of f(w) over the sphere by adaptive quadrature."""
    return integrate.dblquad(lambda ph, th: f(sph(th, ph)) * math.sin(th), 0, math.pi, -math.pi, math.pi,
                             epsabs=eps, epsrel=eps)[0]


def env_from(fn, h=64, w=128):
    d = texel_centres(h, w)
    return np.ascontiguousarray(np.stack([fn(d)] * 3, -1), np.float32)


def test_irradiance_of_constant_and_sky_environments():
    c = np.float32(1.75)
    m = oracle.relight_maps(np.full((64, 128, 3), c, np.float32))
    np.testing.assert_allclose(m["irr"], c, rtol=2e-3)
    # E = max(0, w_z): Irr(N) = 1/pi int max(0, w_z) max(0, w.N) dw, by quadrature
    sky = env_from(lambda d: np.maximum(d[..., 2], 0.0))
    irr = oracle.relight_maps(sky)["irr"]
    cen = texel_centres(32, 64)
    for (i, j) in [(0, 0), (5, 17), (15, 40), (16, 3), (24, 50), (31, 63)]:
        N = cen[i, j]
        ref = sphere_quad(lambda w: max(w[2], 0.0) * max(float(w @ N), 0.0)) / math.pi
        assert abs(irr[i, j, 0] - ref) < 3e-3, (i, j, irr[i, j, 0], ref)
    assert irr[0, 0, 0] > 0.6 and irr[31, 0, 0] < 1e-3       # facing up ~2/3, facing down ~0


def ggx_d(rho, nh):
    a2 = rho ** 4
    q = nh * nh * (a2 - 1) + 1
    return a2 / (math.pi * q * q)


def test_prefilter_constant_exact_and_linear_environment_by_quadrature():
    m = oracle.relight_maps(np.full((32, 64, 3), 2.5, np.float32))
    np.testing.assert_allclose(m["pref"], 2.5, rtol=1e-12)
    lin = env_from(lambda d: 1.0 + d[..., 2])
    pref = oracle.relight_maps(lin)["pref"]
    cen = texel_centres(64, 128)
    for lvl, (i, j) in [(1, (10, 20)), (2, (30, 70)), (3, (50, 5)), (5, (20, 100))]:
        rho = lvl / 5
        R = cen[i, j]

        def wgt(w):
            cs = float(w @ R)
            if cs <= 0:
                return 0.0
            h = (w + R) / np.linalg.norm(w + R)
            return ggx_d(rho, float(h @ R)) * cs
        num = sphere_quad(lambda w: (1 + w[2]) * wgt(w), 1e-6)
        den = sphere_quad(wgt, 1e-6)
        assert abs(pref[lvl - 1, i, j, 0] - num / den) < 4e-3, (lvl, i, j, pref[lvl - 1, i, j, 0], num / den)


def lut_quad(mu, rho, F0part):
    ag = rho * rho
    k = ag / 2
    v = np.array([math.sqrt(1 - mu * mu), 0.0, mu])

    def f(ph, th):
        w = sph(th, ph)
        h = (w + v) / np.linalg.norm(w + v)
        vh = float(v @ h)
        G = (w[2] / (w[2] * (1 - k) + k)) * (mu / (mu * (1 - k) + k))
        fc = (1 - vh) ** 5
        fr = (1 - fc) if F0part else fc
        return ggx_d(rho, h[2]) * G / (4 * mu) * fr * math.sin(th)
    return integrate.dblquad(f, 0, math.pi / 2, 0, 2 * math.pi, epsabs=1e-8, epsrel=1e-7)[0]


@pytest.mark.parametrize("i,j", [(16, 31), (28, 20), (8, 12), (3, 25), (20, 6)])
def test_lut_matches_quadrature_of_the_brdf_integral(i, j):
    lut = oracle.relight_maps(np.ones((4, 8, 3), np.float32))["lut"]
    mu, rho = (i + 0.5) / 32, (j + 0.5) / 32
    A, B = lut_quad(mu, rho, True), lut_quad(mu, rho, False)
    assert abs(lut[i, j, 0] - A) < 4e-3 * max(1.0, A), (A, lut[i, j, 0])
    assert abs(lut[i, j, 1] - B) < 4e-3 * max(1.0, B), (B, lut[i, j, 1])


def test_lut_energy_bound():
    lut = oracle.relight_maps(np.ones((4, 8, 3), np.float32))["lut"]
    assert np.all(lut >= 0) and np.all(lut.sum(-1) <= 1.0 + 2e-3)


def test_environment_sampler_follows_texel_weights():
    rng = np.random.default_rng(4)
    env = rng.uniform(0.1, 5.0, size=(8, 16, 3)).astype(np.float32)
    env[2, 5] = 40.0
    m = oracle.relight_maps(env)
    lum = env @ np.array([0.2126, 0.7152, 0.0722])
    w = lum * np.sin((np.arange(8)[:, None] + 0.5) * math.pi / 8)
    np.testing.assert_allclose(m["row_cdf"][-1], w.sum(), rtol=1e-12)
    np.testing.assert_allclose(np.diff(m["col_cdf"], axis=1), w, rtol=1e-9, atol=1e-12)
    dirs, pdf = oracle.env_samples(env, 4, 50_000, 11)
    d = dirs.reshape(-1, 3)
    th = np.arccos(np.clip(d[:, 2], -1, 1))
    ph = np.arctan2(d[:, 1], d[:, 0])
    row = np.minimum((th / math.pi * 8).astype(int), 7)
    col = np.minimum(((ph + math.pi) / (2 * math.pi) * 16).astype(int), 15)
    freq = np.bincount(row * 16 + col, minlength=128) / d.shape[0]
    p = (w / w.sum()).reshape(-1)
    assert np.all(np.abs(freq - p) < 5 * np.sqrt(p / d.shape[0]) + 1e-4)
    # inside its texel a direction is uniform in (phi, theta)
    for t in (th / math.pi * 8 - row, (ph + math.pi) / (2 * math.pi) * 16 - col):
        assert abs(t.mean() - 0.5) < 0.005 and abs(((t >= 0.25) & (t < 0.75)).mean() - 0.5) < 0.005
    # the pdf is a density on the sphere: E[1/pdf] = 4 pi
    inv = 1.0 / pdf.reshape(-1)
    assert abs(inv.mean() - 4 * math.pi) < 5 * inv.std() / math.sqrt(inv.size)


def spec_albedo(rough, cos_o, F0=0.04):
    ag = rough * rough
    k = ag / 2
    wo = np.array([math.sqrt(1 - cos_o ** 2), 0.0, cos_o])

    def f(ph, th):
        wi = sph(th, ph)
        h = (wi + wo) / np.linalg.norm(wi + wo)
        ni = wi[2]
        F = F0 + (1 - F0) * (1 - float(wo @ h)) ** 5
        G = (ni / (ni * (1 - k) + k)) * (cos_o / (cos_o * (1 - k) + k))
        return ggx_d(rough, h[2]) * F * G / (4 * ni * cos_o) * ni * math.sin(th)
    return integrate.dblquad(f, 0, math.pi / 2, 0, 2 * math.pi, epsabs=1e-8, epsrel=1e-7)[0]


def _empty():
    z = np.zeros((0, 3), np.float32)
    return scene(z, np.zeros((0, 4)), np.zeros((0, 2)), np.zeros(0), np.zeros((0, 7)))


def test_relight_furnace_in_an_empty_scene():
    P, rough, th = 64, 0.5, 25.0
    co = math.cos(math.radians(th))
    wo = np.tile(np.array([math.sqrt(1 - co * co), 0, co], np.float32), (P, 1))
    x = np.zeros((P, 3), np.float32)
    n = np.tile(np.array([0, 0, 1.0], np.float32), (P, 1))
    a = np.tile(np.array([0.3, 0.5, 0.7], np.float32), (P, 1))
    r = np.full(P, rough, np.float32)
    L = np.array([1.5, 1.0, 0.5], np.float32)
    env = np.tile(L, (16, 32, 1)).astype(np.float32)
    out = oracle.relight(_empty(), x, n, a, r, wo, env, 256, 17, PR)
    ref = L.astype(np.float64) * (a[0].astype(np.float64) + spec_albedo(rough, co))
    for c in range(3):
        est = out["rgb"][:, c]
        sem = est.std(ddof=1) / math.sqrt(P)
        assert abs(est.mean() - ref[c]) < 4.5 * sem + 1e-4, (c, est.mean(), ref[c], sem)
    np.testing.assert_allclose(out["vis"], 1.0)
    np.testing.assert_allclose(out["ind"], 0.0)


def canopy(albedo):
    """One large opaque surfel above the origin, facing down; material
    channels [a (3), r, n (3)]."""
    means = np.array([[0.0, 0.0, 1.0]], np.float32)
    quats = np.array([[0.0, 1.0, 0.0, 0.0]], np.float32)       # 180 deg about x: normal -z
    feats = np.array([[albedo, albedo, albedo, 0.6, 0.0, 0.0, -1.0]], np.float32)
    # wide enough that alpha = alpha_max up to 0.004 deg above the horizon
    return scene(means, quats, np.array([[1e5, 1e5]]), np.array([1.0]), feats)


def test_relight_indirect_diffuse_part_and_visibility_under_an_opaque_canopy():
    """Two canopies that differ only in albedo: the specular part of L_ind
    and every sample cancel in the difference, which must be
    O * (a1 - a0) * Irr * (fraction of samples that hit the canopy), with
    Irr = c for a constant environment and O = alpha_max."""
    P = 8
    x = np.zeros((P, 3), np.float32)
    n = np.tile(np.array([0, 0, 1.0], np.float32), (P, 1))
    wo = np.tile(np.array([0.0, 0.0, 1.0], np.float32), (P, 1))
    a = np.full((P, 3), 0.5, np.float32)
    r = np.full(P, 0.5, np.float32)
    c = 1.25
    env = np.full((16, 32, 3), c, np.float32)
    S = 128
    o0 = oracle.relight(canopy(0.0), x, n, a, r, wo, env, S, 23, PR)
    o1 = oracle.relight(canopy(0.8), x, n, a, r, wo, env, S, 23, PR)
    dirs, _ = oracle.env_samples(env, P, S, 23)
    up = (dirs[..., 2] > 0).mean(1)                 # samples that reach the canopy
    irr = oracle.relight_maps(env)["irr"][-1].mean()      # the map's bottom row: normal -z
    assert abs(irr - c) < 1e-2 * c                        # 16-row texel sum
    np.testing.assert_allclose(o1["ind"][:, 0] - o0["ind"][:, 0], 0.99 * 0.8 * irr * up, rtol=1e-3)
    np.testing.assert_allclose(o0["vis"], 1.0 - 0.99 * up, rtol=1e-9)
