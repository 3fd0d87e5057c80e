"""Pins of the oracle's analytic gradient: FP64 central finite differences of
the oracle's own (separately pinned) forward, plus single-surfel closed forms.

Inputs are float32, so each perturbation is rounded to float32 and the exact
step (theta_plus - theta_minus) is used as the denominator.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from oracle import Params, Margins
import synth
from tests.helpers import frame_of, quat_wxyz, rays, scene

PG = Params(alpha_min=1 / 255, alpha_max=0.99, T_min=1e-4, feat_offset=0, feat_count=3)
WIDE = Margins(alpha_abs=2e-3, rho_rel=2e-2, T_rel=2e-2, tie_abs=2e-3, t_abs=1e-3, clamp_abs=2e-3)


def _loss(sc, ro, rd, gf, gd, go, p):
    out = oracle.trace(sc, ro, rd, p, margins=None)
    return float(np.sum(out["feat"] * gf) + np.sum(out["depth"] * gd) + np.sum(out["opacity"] * go))


def _fd_check(sc, ro, rd, p, rel_tol=2e-4, seed=0):
    rng = np.random.default_rng(seed)
    R = ro.shape[0]
    gf = rng.normal(size=(R, p.feat_count)).astype(np.float32)
    gd = rng.normal(size=R).astype(np.float32)
    go = rng.normal(size=R).astype(np.float32)
    ana = oracle.trace_grad(sc, ro, rd, gf, gd, go, p)
    names = ["means", "quats", "scales", "opacity", "features"]
    worst = 0.0
    for name in names:
        arr = getattr(sc, name)
        g_ana = ana[name].reshape(arr.shape)
        flat = arr.reshape(-1)
        g_fd = np.zeros(flat.shape[0])
        for i in range(flat.shape[0]):
            x0 = float(flat[i])
            h = 3e-4 * max(abs(x0), 0.05 if name != "means" else 1.0)
            xp, xm = np.float32(x0 + h), np.float32(x0 - h)
            flat[i] = xp
            lp = _loss(sc, ro, rd, gf, gd, go, p)
            flat[i] = xm
            lm = _loss(sc, ro, rd, gf, gd, go, p)
            flat[i] = np.float32(x0)
            g_fd[i] = (lp - lm) / (float(xp) - float(xm))
        g_a = g_ana.reshape(-1)
        scale = max(np.abs(g_fd).max(), 1e-12)
        err = np.abs(g_a - g_fd).max() / scale
        worst = max(worst, err)
        assert err < rel_tol, (name, err, np.c_[g_a, g_fd][np.argsort(-np.abs(g_a - g_fd))[:4]])
    return worst


def _clean_rays(sc, ro, rd, p):
    out = oracle.trace(sc, ro, rd, p, margins=WIDE)
    ok = (out["flags"] == 0) & (out["n_hits"] > 0)
    return ro[ok], rd[ok]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(100 + seed)
    n = 10
    sc = synth.tiny_scene(seed=100 + seed, n=n)
    # spread them around the origin, large enough to overlap along rays
    sc.means[:] = (rng.uniform(-0.4, 0.4, size=(n, 3))).astype(np.float32)
    sc.scales[:] = np.exp(rng.uniform(math.log(0.15), math.log(0.4), size=(n, 2))).astype(np.float32)
    # unnormalised quaternions exercise the normalisation chain
    sc.quats[:] = (sc.quats * rng.uniform(0.5, 2.0, size=(n, 1))).astype(np.float32)
    sc.opacity[:] = rng.uniform(0.2, 0.9, size=n).astype(np.float32)
    ro, rd = synth.random_rays_through_scene(80, seed=200 + seed, box=0.4)
    ro, rd = _clean_rays(sc, ro, rd, PG)
    assert ro.shape[0] >= 30
    _fd_check(sc, ro, rd, PG, seed=seed)


def test_gradient_with_clamp_and_termination():
    # opaque stack: alpha clamped for some, T_min termination reached
    rng = np.random.default_rng(5)
    n = 8
    sc = synth.tiny_scene(seed=55, n=n)
    sc.means[:] = rng.uniform(-0.2, 0.2, size=(n, 3)).astype(np.float32)
    sc.scales[:] = rng.uniform(0.3, 0.5, size=(n, 2)).astype(np.float32)
    sc.opacity[:] = rng.uniform(0.85, 0.999, size=n).astype(np.float32)
    p = Params(alpha_min=1 / 255, alpha_max=0.99, T_min=1e-3, feat_offset=0, feat_count=3)
    ro, rd = synth.random_rays_through_scene(60, seed=56, box=0.15)
    ro, rd = _clean_rays(sc, ro, rd, p)
    assert ro.shape[0] >= 20
    _fd_check(sc, ro, rd, p, seed=9)


def test_single_surfel_closed_form_gradients():
    q = quat_wxyz(Rotation.from_rotvec([0.3, 0.2, -0.4]))
    tu, tv, n = frame_of(q)
    su, sv = 0.2, 0.3
    a, b = 0.8, -0.5
    sc = scene([0, 0, 0], q, [su, sv], [0.6], [0.1, 0.2, 0.3])
    s32 = sc.scales[0].astype(np.float64)
    p0 = a * s32[0] * tu + b * s32[1] * tv
    ro, rd = rays(p0 + 2 * n, -n)
    o32 = float(sc.opacity[0])
    G = math.exp(-(a * a + b * b) / 2)
    alpha = o32 * G
    # dO/dopacity = G ; dO/ds_u = alpha u^2 / s_u
    g = oracle.trace_grad(sc, ro, rd, np.zeros((1, 3), np.float32), np.zeros(1, np.float32),
                          np.ones(1, np.float32), PG)
    np.testing.assert_allclose(g["opacity"][0], G, rtol=1e-6)
    np.testing.assert_allclose(g["scales"][0, 0], alpha * a * a / s32[0], rtol=1e-5)
    np.testing.assert_allclose(g["scales"][0, 1], alpha * b * b / s32[1], rtol=1e-5)
    # dC/df = alpha g_C
    gC = np.array([[1.0, -2.0, 0.5]], np.float32)
    g = oracle.trace_grad(sc, ro, rd, gC, np.zeros(1, np.float32), np.zeros(1, np.float32), PG)
    np.testing.assert_allclose(g["features"][0], alpha * gC[0], rtol=1e-6)
    # a clamped surfel passes no gradient to its opacity
    sc2 = scene([0, 0, 0], q, [su, sv], [0.999], [0.1, 0.2, 0.3])
    ro2, rd2 = rays(2 * n, -n)
    g = oracle.trace_grad(sc2, ro2, rd2, np.zeros((1, 3), np.float32), np.zeros(1, np.float32),
                          np.ones(1, np.float32), PG)
    assert g["opacity"][0] == 0.0


def test_gradient_translation_equivariance():
    # moving every surfel by the same offset and the ray origin with it leaves
    # the loss unchanged, so the mean gradients of the hit surfels plus the
    # (implicit) origin gradient sum to zero: check with the moved origin FD.
    sc = synth.tiny_scene(seed=77, n=6)
    sc.means[:] *= 0.2
    sc.scales[:] = 0.3
    ro, rd = synth.random_rays_through_scene(30, seed=78, box=0.2)
    ro, rd = _clean_rays(sc, ro, rd, PG)
    rng = np.random.default_rng(1)
    R = ro.shape[0]
    gf = rng.normal(size=(R, 3)).astype(np.float32)
    gd = rng.normal(size=R).astype(np.float32)
    go = rng.normal(size=R).astype(np.float32)
    g = oracle.trace_grad(sc, ro, rd, gf, gd, go, PG)
    total = g["means"].sum(axis=0)
    # d loss / d origin (all rays moved along axis k) must equal -total;
    # per-ray float32 steps, so take the per-ray difference quotients
    def per_ray(r_o):
        out = oracle.trace(sc, r_o, rd, PG, margins=None)
        return (out["feat"] * gf).sum(1) + out["depth"] * gd + out["opacity"] * go
    for k in range(3):
        rp, rm = ro.copy(), ro.copy()
        rp[:, k] += np.float32(1e-3)
        rm[:, k] -= np.float32(1e-3)
        step = rp[:, k].astype(np.float64) - rm[:, k].astype(np.float64)
        dl = ((per_ray(rp) - per_ray(rm)) / step).sum()
        np.testing.assert_allclose(dl, -total[k], rtol=2e-3, atol=1e-6)
