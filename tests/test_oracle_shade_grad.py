"""Pins of the oracle's stratified-uniform estimator (Eq. 15) and of its
shading gradient (sample directions held fixed).

* albedo and environment enter linearly: the gradient equals the difference
  quotient exactly;
* with uniform sampling the directions do not depend on roughness or on the
  surfels, so central differences of the oracle's own estimate pin the
  roughness and surfel gradients;
* with GGX sampling the roughness gradient is checked for unbiasedness
  against the derivative of an adaptive-quadrature specular albedo;
* the uniform estimator converges to the diffuse + specular albedo furnace.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import MODE_SPLIT, MODE_UNIFORM, Margins, Params
from tests.helpers import scene

PS = Params(alpha_min=1 / 255, alpha_max=0.99, T_min=1e-4, t_min=1e-3, feat_offset=0, feat_count=3)
# margins wide enough for a 2e-4 relative parameter step
FD_MARGINS = Margins(alpha_abs=1e-4, rho_rel=2e-3, T_rel=1e-3, tie_abs=1e-4, t_abs=1e-4, clamp_abs=1e-4)


def canopy():
    """A few large tilted surfels above points on the z = 0 plane."""
    rng = np.random.default_rng(3)
    m = 6
    means = np.c_[rng.uniform(-0.6, 0.6, m), rng.uniform(-0.6, 0.6, m), rng.uniform(0.4, 1.2, m)]
    q = rng.normal(size=(m, 4))
    q[:, 0] += 4.0                      # mostly facing down/up
    feats = rng.uniform(0.2, 1.0, size=(m, 3))
    return scene(means, q, rng.uniform(0.3, 0.6, size=(m, 2)), rng.uniform(0.3, 0.8, m), feats)


def points(P=3, seed=4):
    rng = np.random.default_rng(seed)
    x = np.c_[rng.uniform(-0.3, 0.3, P), rng.uniform(-0.3, 0.3, P), np.zeros(P)].astype(np.float32)
    n = np.tile(np.array([0, 0, 1.0], np.float32), (P, 1))
    wo = np.c_[rng.uniform(-0.4, 0.4, P), rng.uniform(-0.4, 0.4, P), np.ones(P)]
    wo = (wo / np.linalg.norm(wo, axis=1, keepdims=True)).astype(np.float32)
    a = rng.uniform(0.2, 0.8, size=(P, 3)).astype(np.float32)
    r = rng.uniform(0.3, 0.8, size=P).astype(np.float32)
    return x, n, a, r, wo


def env_small(seed=5):
    return np.random.default_rng(seed).uniform(0.5, 3.0, size=(8, 16, 3)).astype(np.float32)


def loss(sc, x, n, a, r, wo, env, nd, ns, mode, g, seed=9):
    o = oracle.shade(sc, x, n, a, r, wo, env, nd, ns, seed, PS, margins=None, mode=mode)
    return float((o["rgb"] * g).sum())


@pytest.mark.parametrize("mode,nd,ns", [(MODE_SPLIT, 6, 5), (MODE_UNIFORM, 9, 0)])
def test_albedo_and_env_gradients_are_exact_difference_quotients(mode, nd, ns):
    sc = canopy()
    x, n, a, r, wo = points()
    env = env_small()
    g = np.random.default_rng(1).normal(size=(x.shape[0], 3)).astype(np.float32)
    gr = oracle.shade_grad(sc, x, n, a, r, wo, env, nd, ns, 9, PS, g, mode=mode)
    for p in range(x.shape[0]):
        for c in range(3):
            ap, am = a.copy(), a.copy()
            ap[p, c] += np.float32(0.125)
            am[p, c] -= np.float32(0.125)
            step = float(ap[p, c]) - float(am[p, c])
            fd = (loss(sc, x, n, ap, r, wo, env, nd, ns, mode, g) - loss(sc, x, n, am, r, wo, env, nd, ns, mode, g)) / step
            np.testing.assert_allclose(gr["albedo"][p, c], fd, rtol=1e-9, atol=1e-12)
    hot = np.argsort(-np.abs(gr["env"]).reshape(-1))[:6]
    for i in hot:
        e1, e2 = env.copy().reshape(-1), env.copy().reshape(-1)
        e1[i] += np.float32(0.5)
        e2[i] -= np.float32(0.5)
        step = float(e1[i]) - float(e2[i])
        fd = (loss(sc, x, n, a, r, wo, e1.reshape(env.shape), nd, ns, mode, g)
              - loss(sc, x, n, a, r, wo, e2.reshape(env.shape), nd, ns, mode, g)) / step
        np.testing.assert_allclose(gr["env"].reshape(-1)[i], fd, rtol=1e-8, atol=1e-12)


def test_uniform_roughness_gradient_matches_central_differences():
    sc = canopy()
    x, n, a, r, wo = points()
    env = env_small()
    g = np.random.default_rng(2).normal(size=(x.shape[0], 3)).astype(np.float32)
    gr = oracle.shade_grad(sc, x, n, a, r, wo, env, 16, 0, 9, PS, g, mode=MODE_UNIFORM)
    for p in range(x.shape[0]):
        rp, rm = r.copy(), r.copy()
        h = 1e-4            # D ~ r^-4 near the peak: keep the truncation error small
        rp[p] = np.float32(r[p] + h)
        rm[p] = np.float32(r[p] - h)
        fd = (loss(sc, x, n, a, rp, wo, env, 16, 0, MODE_UNIFORM, g)
              - loss(sc, x, n, a, rm, wo, env, 16, 0, MODE_UNIFORM, g)) / (float(rp[p]) - float(rm[p]))
        np.testing.assert_allclose(gr["rough"][p], fd, rtol=2e-5, atol=1e-9)


@pytest.mark.parametrize("mode,nd,ns", [(MODE_SPLIT, 8, 8), (MODE_UNIFORM, 12, 0)])
def test_surfel_gradients_through_traced_rays(mode, nd, ns):
    sc = canopy()
    x, n, a, r, wo = points(P=16)
    env = env_small()
    f = oracle.shade(sc, x, n, a, r, wo, env, nd, ns, 9, PS, margins=FD_MARGINS, mode=mode)
    keep = f["flags"] == 0
    assert keep.sum() >= 4
    x, n, a, r, wo = (v[keep] for v in (x, n, a, r, wo))
    pid = np.nonzero(keep)[0]
    g = np.random.default_rng(3).normal(size=(x.shape[0], 3)).astype(np.float32)
    gr = oracle.shade_grad(sc, x, n, a, r, wo, env, nd, ns, 9, PS, g, mode=mode, point_ids=pid)

    def L():
        o = oracle.shade(sc, x, n, a, r, wo, env, nd, ns, 9, PS, margins=None, mode=mode, point_ids=pid)
        return float((o["rgb"] * g).sum())

    total = 0.0
    for name in ("means", "quats", "scales", "opacity", "features"):
        arr = getattr(sc, name)
        flat = arr.reshape(-1)
        fd = np.zeros(flat.size)
        for i in range(flat.size):
            x0 = float(flat[i])
            h = 2e-4 * max(abs(x0), 0.1)
            flat[i] = np.float32(x0 + h); lp = L(); xp = float(flat[i])
            flat[i] = np.float32(x0 - h); lm = L(); xm = float(flat[i])
            flat[i] = np.float32(x0)
            fd[i] = (lp - lm) / (xp - xm)
        ana = gr[name].reshape(-1)[: flat.size] if name != "features" else gr[name][:, :3].reshape(-1)
        scale = max(np.abs(fd).max(), 1e-9)
        assert np.abs(ana - fd).max() / scale < 5e-4, (name, np.c_[ana, fd][:6])
        total += np.abs(fd).sum()
    assert total > 0.0


def _spec_albedo(rough, cos_o, F0=0.04):
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

    return integrate.dblquad(f, 0, 2 * math.pi, 0, math.pi / 2, epsabs=1e-8, epsrel=1e-7)[0]


def _empty():
    z = np.zeros((0, 3), np.float32)
    return scene(z, np.zeros((0, 4)), np.zeros((0, 2)), np.zeros(0), np.zeros((0, 3)))


def test_ggx_roughness_gradient_is_unbiased():
    P, rough, th = 48, 0.6, 35.0
    co = math.cos(math.radians(th))
    wo = np.tile(np.array([math.sqrt(1 - co * co), 0, co], np.float32), (P, 1))
    x = np.zeros((P, 3), np.float32)
    n = np.tile(np.array([0, 0, 1.0], np.float32), (P, 1))
    a = np.zeros((P, 3), np.float32)
    r = np.full(P, rough, np.float32)
    env = np.ones((8, 16, 3), np.float32)
    g = np.zeros((P, 3), np.float32)
    g[:, 0] = 1.0
    gr = oracle.shade_grad(_empty(), x, n, a, r, wo, env, 0, 1024, 21, PS, g)["rough"]
    r0 = float(r[0])
    ref = (_spec_albedo(r0 + 1e-4, float(wo[0, 2])) - _spec_albedo(r0 - 1e-4, float(wo[0, 2]))) / 2e-4
    sem = gr.std(ddof=1) / math.sqrt(P)
    assert abs(gr.mean() - ref) < 4.5 * sem + 1e-5, (gr.mean(), ref, sem)


def test_uniform_estimator_furnace():
    P, rough, th = 48, 0.5, 20.0
    co = math.cos(math.radians(th))
    wo = np.tile(np.array([math.sqrt(1 - co * co), 0, co], np.float32), (P, 1))
    x = np.zeros((P, 3), np.float32)
    n = np.tile(np.array([0, 0, 1.0], np.float32), (P, 1))
    a = np.tile(np.array([0.3, 0.5, 0.7], np.float32), (P, 1))
    r = np.full(P, rough, np.float32)
    L = np.array([1.5, 1.0, 0.5], np.float32)
    env = np.tile(L, (8, 16, 1)).astype(np.float32)
    out = oracle.shade(_empty(), x, n, a, r, wo, env, 256, 0, 33, PS, mode=MODE_UNIFORM)
    ref = L.astype(np.float64) * (a[0].astype(np.float64) + _spec_albedo(float(r[0]), float(wo[0, 2])))
    for c in range(3):
        est = out["rgb"][:, c]
        sem = est.std(ddof=1) / math.sqrt(P)
        assert abs(est.mean() - ref[c]) < 4.5 * sem + 1e-4, (c, est.mean(), ref[c], sem)
    np.testing.assert_allclose(out["vis"], 1.0)


def test_uniform_directions_are_stratified_in_cos_theta():
    nrm = np.array([[0.2, -0.3, 0.9]], np.float32)
    dirs, valid = oracle.sample_dirs(nrm, nrm, np.array([0.5], np.float32), 64, 0, 3, mode=MODE_UNIFORM)
    nn = nrm[0].astype(np.float64) / np.linalg.norm(nrm[0])
    z = dirs[0] @ nn
    assert valid.all()
    np.testing.assert_array_equal(np.floor(z * 64).astype(int), np.arange(64))
