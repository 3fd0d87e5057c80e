"""Pins of the FP64 oracle's forward trace (Eq. 2, 6-8) against closed forms,
an independent linear-solve formulation, invariants and textbook routines.

None of these tests re-types the oracle's own formula: the frame comes from
SciPy's rotation matrix, hit points from a 3x3 linear solve, and blending
from closed-form products.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from oracle import Params, Margins
import synth
from tests.helpers import frame_of, quat_wxyz, rays, scene

P0 = Params(alpha_min=1 / 255, alpha_max=0.99, T_min=1e-4, t_min=0.0, t_max=math.inf,
            feat_offset=0, feat_count=3)


def one(sc, o, d, params=P0, **kw):
    ro, rd = rays(o, d)
    return oracle.trace(sc, ro, rd, params, **kw)


def test_single_surfel_center_hit_alpha_is_opacity():
    q = quat_wxyz(Rotation.from_euler("xyz", [0.3, -0.7, 1.1]))
    _, _, n = frame_of(q)
    mu = np.array([0.3, -0.2, 0.5])
    f = np.array([0.2, 0.5, 0.9])
    sc = scene(mu, q, [0.05, 0.1], [0.7], f)
    o32 = sc.opacity[0].astype(np.float64)
    out = one(sc, mu + 2.5 * n, -n)
    assert out["n_hits"][0] == 1
    # tau = distance along the normal; alpha = opacity at the centre
    np.testing.assert_allclose(out["opacity"][0], o32, rtol=0, atol=1e-6)
    np.testing.assert_allclose(out["feat"][0], o32 * sc.features[0].astype(np.float64), atol=1e-6)
    np.testing.assert_allclose(out["depth"][0], o32 * 2.5, atol=1e-5)


def test_alpha_clamped_at_alpha_max():
    q = quat_wxyz(Rotation.identity())
    sc = scene([0, 0, 0], q, [0.1, 0.1], [0.995], [1, 1, 1])
    out = one(sc, [0, 0, 3], [0, 0, -1])
    np.testing.assert_allclose(out["opacity"][0], 0.99, atol=1e-12)


@pytest.mark.parametrize("a,b", [(0.7, -1.3), (-1.9, 0.4), (0.0, 2.2)])
def test_offset_hit_gaussian_falloff(a, b):
    q = quat_wxyz(Rotation.from_rotvec([0.4, 0.9, -0.2]))
    tu, tv, n = frame_of(q)
    su, sv = 0.03, 0.11
    mu = np.array([-0.4, 0.1, 0.2])
    sc = scene(mu, q, [su, sv], [0.8], [1, 0, 0])
    s32 = sc.scales[0].astype(np.float64)
    p = mu + a * s32[0] * tu + b * s32[1] * tv
    out = one(sc, p + 1.7 * n, -n)
    expect = float(sc.opacity[0]) * math.exp(-(a * a + b * b) / 2)
    np.testing.assert_allclose(out["opacity"][0], expect, rtol=2e-6)


def test_two_parallel_surfels_blend_front_to_back():
    q = quat_wxyz(Rotation.from_rotvec([0.2, -0.1, 0.3]))
    _, _, n = frame_of(q)
    mu1 = np.zeros(3)
    mu2 = mu1 - 0.5 * n
    f1, f2 = np.array([1.0, 0.0, 0.25]), np.array([0.0, 1.0, 0.5])
    sc = scene([mu1, mu2], [q, q], [[0.2, 0.2]] * 2, [0.6, 0.5], [f1, f2])
    a1, a2 = (float(x) for x in sc.opacity)
    front = one(sc, mu1 + 2 * n, -n)
    np.testing.assert_allclose(front["feat"][0], a1 * f1 + (1 - a1) * a2 * f2, atol=1e-6)
    np.testing.assert_allclose(front["opacity"][0], 1 - (1 - a1) * (1 - a2), atol=1e-7)
    back = one(sc, mu2 - 2 * n, n)
    np.testing.assert_allclose(back["feat"][0], a2 * f2 + (1 - a2) * a1 * f1, atol=1e-6)
    np.testing.assert_allclose(back["depth"][0], a2 * 2.0 + (1 - a2) * a1 * 2.5, atol=1e-5)


def test_ray_parallel_to_disk_misses():
    q = quat_wxyz(Rotation.identity())
    sc = scene([0, 0, 0], q, [0.5, 0.5], [0.9], [1, 1, 1])
    out = one(sc, [-3, 0, 0], [1, 0, 0])
    assert out["n_hits"][0] == 0 and out["opacity"][0] == 0.0
    # nearly parallel (|n.d| below 1e-8 |d|) also misses
    d = np.array([1.0, 0.0, 1e-9])
    out = one(sc, [-3, 0, 3e-9], d)
    assert out["n_hits"][0] == 0


def test_coincident_stack_termination_rule():
    # m identical surfels along z, alpha = 0.8: (0.2)^5 = 3.2e-4 >= 1e-4 and
    # (0.2)^6 = 6.4e-5 < 1e-4, so the sixth hit is included and the march stops.
    q = quat_wxyz(Rotation.identity())
    m = 10
    mus = [[0, 0, -0.1 * i] for i in range(m)]
    sc = scene(mus, [q] * m, [[0.2, 0.2]] * m, [0.8] * m, np.tile([1.0, 0.5, 0.25], (m, 1)))
    a = float(sc.opacity[0])
    out = one(sc, [0, 0, 1], [0, 0, -1])
    assert out["n_hits"][0] == 6
    np.testing.assert_allclose(out["opacity"][0], 1 - (1 - a) ** 6, rtol=1e-12)
    # without early termination all m are blended
    out = one(sc, [0, 0, 1], [0, 0, -1], Params(T_min=0.0))
    assert out["n_hits"][0] == m
    np.testing.assert_allclose(out["opacity"][0], 1 - (1 - a) ** m, rtol=1e-12)


@pytest.mark.parametrize("opac", [0.9, 0.05])
def test_support_cut_radius(opac):
    # rho_c = min(3, sqrt(2 ln(o/alpha_min)))
    q = quat_wxyz(Rotation.identity())
    sc = scene([0, 0, 0], q, [0.1, 0.1], [opac], [1, 1, 1])
    o32 = float(sc.opacity[0])
    s = float(sc.scales[0, 0])
    rc = min(3.0, math.sqrt(2 * math.log(o32 / (1 / 255))))
    inside = one(sc, [0.999 * rc * s, 0, 1], [0, 0, -1])
    outside = one(sc, [1.001 * rc * s, 0, 1], [0, 0, -1])
    assert inside["n_hits"][0] == 1 and outside["n_hits"][0] == 0


def test_opacity_below_cutoff_never_hits():
    q = quat_wxyz(Rotation.identity())
    sc = scene([0, 0, 0], q, [0.1, 0.1], [0.003], [1, 1, 1])
    assert one(sc, [0, 0, 1], [0, 0, -1])["n_hits"][0] == 0


def test_ray_interval_is_open():
    q = quat_wxyz(Rotation.identity())
    sc = scene([0, 0, 0], q, [0.1, 0.1], [0.5], [1, 1, 1])
    o, d = [0, 0, 0.5], [0, 0, -1]
    assert one(sc, o, d, Params(t_min=0.4))["n_hits"][0] == 1
    assert one(sc, o, d, Params(t_min=0.6))["n_hits"][0] == 0
    assert one(sc, o, d, Params(t_max=0.6))["n_hits"][0] == 1
    assert one(sc, o, d, Params(t_max=0.4))["n_hits"][0] == 0
    # behind the origin never counts with t_min = 0
    assert one(sc, [0, 0, -0.5], d)["n_hits"][0] == 0


def test_equal_depth_tie_broken_by_user_index():
    q = quat_wxyz(Rotation.identity())
    fa, fb = [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]
    sc = scene([[0, 0, 0]] * 2, [q, q], [[0.1, 0.1]] * 2, [0.5, 0.5], [fa, fb])
    out = one(sc, [0, 0, 1], [0, 0, -1], max_ids=4)
    assert list(out["ids"][0, :2]) == [0, 1]
    np.testing.assert_allclose(out["feat"][0], [0.5, 0.25, 0.0], atol=1e-12)
    sc2 = scene([[0, 0, 0]] * 2, [q, q], [[0.1, 0.1]] * 2, [0.5, 0.5], [fb, fa])
    np.testing.assert_allclose(one(sc2, [0, 0, 1], [0, 0, -1])["feat"][0], [0.25, 0.5, 0.0], atol=1e-12)


def test_depth_units_of_direction_length():
    q = quat_wxyz(Rotation.identity())
    sc = scene([0, 0, 0], q, [0.1, 0.1], [0.5], [1, 1, 1])
    out = one(sc, [0, 0, 2], [0, 0, -2])   # |d| = 2: tau = 1
    np.testing.assert_allclose(out["depth"][0], 0.5 * 1.0, atol=1e-12)


def _linear_solve_reference(sc, ro, rd, params):
    """Independent brute force: hit point from the 3x3 system
    o + tau d = mu + (u s_u) t_u + (v s_v) t_v, frame from SciPy."""
    means = sc.means.astype(np.float64)
    scales = sc.scales.astype(np.float64)
    op = sc.opacity.astype(np.float64)
    feats = sc.features.astype(np.float64)[:, params.feat_offset:params.feat_offset + params.feat_count]
    frames = []
    for q in sc.quats.astype(np.float64):
        q = q / np.linalg.norm(q)
        frames.append(frame_of(q))
    res = []
    for o, d in zip(ro.astype(np.float64), rd.astype(np.float64)):
        hits = []
        for i in range(sc.n):
            tu, tv, n = frames[i]
            if abs(n @ d) < 1e-8 * np.linalg.norm(d):
                continue
            A = np.stack([scales[i, 0] * tu, scales[i, 1] * tv, -d], axis=1)
            u, v, tau = np.linalg.solve(A, o - means[i])
            rho2 = u * u + v * v
            rc2 = min(9.0, 2 * math.log(op[i] / params.alpha_min))
            alpha = min(params.alpha_max, op[i] * math.exp(-rho2 / 2))
            if rho2 <= rc2 and alpha >= params.alpha_min and params.t_min < tau < params.t_max:
                hits.append((tau, i, alpha))
        hits.sort()
        T, Cc, D, nh = 1.0, np.zeros(params.feat_count), 0.0, 0
        for tau, i, a in hits:
            Cc += T * a * feats[i]
            D += T * a * tau
            T *= 1 - a
            nh += 1
            if T < params.T_min:
                break
        res.append((Cc, D, 1 - T, nh))
    return res


def test_matches_independent_linear_solve_bruteforce():
    sc = synth.tiny_scene(seed=7, n=48)
    # make the surfels large enough that most rays hit several of them
    sc.scales[:] = sc.scales * 3.0
    ro, rd = synth.random_rays_through_scene(96, seed=8)
    out = oracle.trace(sc, ro, rd, P0)
    ref = _linear_solve_reference(sc, ro, rd, P0)
    clean = (out["flags"] & oracle.FORWARD_FLAGS) == 0
    assert clean.mean() > 0.9
    hits = 0
    for r, (Cc, D, O, nh) in enumerate(ref):
        if not clean[r]:
            continue
        hits += nh
        assert out["n_hits"][r] == nh
        np.testing.assert_allclose(out["feat"][r], Cc, atol=1e-9)
        np.testing.assert_allclose(out["depth"][r], D, atol=1e-9)
        np.testing.assert_allclose(out["opacity"][r], O, atol=1e-9)
    assert hits > 100


def test_invariant_to_surfel_order_and_rigid_motion():
    sc = synth.tiny_scene(seed=11, n=256)
    ro, rd = synth.random_rays_through_scene(512, seed=12)
    base = oracle.trace(sc, ro, rd, P0)
    clean = (base["flags"] & oracle.FORWARD_FLAGS) == 0
    perm = np.random.default_rng(0).permutation(sc.n)
    outp = oracle.trace(sc.subset(perm), ro, rd, P0)
    for k in ("feat", "depth", "opacity"):
        np.testing.assert_allclose(outp[k][clean], base[k][clean], atol=1e-12)
    np.testing.assert_array_equal(outp["n_hits"][clean], base["n_hits"][clean])
    # rigid motion: rotate + translate scene and rays (in float64, then float32)
    rot = Rotation.from_rotvec([0.3, -0.5, 0.8])
    t = np.array([0.25, -0.5, 0.125])
    R = rot.as_matrix()
    q_old = Rotation.from_quat(np.c_[sc.quats[:, 1:], sc.quats[:, :1]].astype(np.float64))
    q_new = (rot * q_old).as_quat()
    sc2 = scene(sc.means.astype(np.float64) @ R.T + t, np.c_[q_new[:, 3:], q_new[:, :3]],
                sc.scales, sc.opacity, sc.features)
    out2 = oracle.trace(sc2, ro.astype(np.float64) @ R.T + t, rd.astype(np.float64) @ R.T, P0)
    clean2 = clean & ((out2["flags"] & oracle.FORWARD_FLAGS) == 0)
    assert clean2.mean() > 0.95
    # float32 re-rounding of the moved inputs bounds the agreement
    np.testing.assert_allclose(out2["opacity"][clean2], base["opacity"][clean2], atol=2e-4)
    np.testing.assert_allclose(out2["feat"][clean2], base["feat"][clean2], atol=2e-4)


def test_output_ranges_on_object_scene():
    sc = synth.object_scene(n=20_000, seed=5)
    cams = synth.hemisphere_cameras(2, seed=5)
    ro, rd = synth.camera_batch_rays(cams, 24, 24)
    p = Params(feat_offset=0, feat_count=10)
    out = oracle.trace(sc, ro, rd, p)
    O = out["opacity"]
    assert np.all(O >= 0) and np.all(O <= 1)
    fmax = sc.features.max(axis=0).astype(np.float64)
    fmin = sc.features.min(axis=0).astype(np.float64)
    assert np.all(out["feat"] <= O[:, None] * fmax + 1e-12)
    assert np.all(out["feat"] >= O[:, None] * np.minimum(fmin, 0) - 1e-12)
    hit = out["n_hits"] > 0
    assert hit.mean() > 0.3
    # normalised depth lies within the camera distance range of the scene
    dn = out["depth"][hit] / O[hit]
    assert np.all(dn > 0.5) and np.all(dn < 9.0)


def test_ids_sorted_by_depth_and_transmittance_monotone():
    sc = synth.tiny_scene(seed=21, n=300)
    sc.scales[:] *= 2.0
    ro, rd = synth.random_rays_through_scene(200, seed=22)
    out = oracle.trace(sc, ro, rd, P0, max_ids=64)
    for r in range(200):
        nh = out["n_hits"][r]
        taus = out["tau"][r, :min(nh, 64)]
        assert np.all(np.diff(taus) >= 0)
    # O grows with more hits (T non-increasing): a prefix of the scene can only see less
    p_sub = sc.subset(np.arange(150))
    out_sub = oracle.trace(p_sub, ro, rd, Params(T_min=0.0))
    out_all = oracle.trace(sc, ro, rd, Params(T_min=0.0))
    assert np.all(out_all["opacity"] >= out_sub["opacity"] - 1e-12)


def test_flags_mark_threshold_neighbourhoods():
    q = quat_wxyz(Rotation.identity())
    sc = scene([0, 0, 0], q, [0.1, 0.1], [0.9], [1, 1, 1])
    # exactly at the 3-sigma cut: flagged
    out = one(sc, [0.3, 0, 1], [0, 0, -1])
    assert out["flags"][0] & oracle.F_RHO
    # well inside: clean
    out = one(sc, [0.1, 0, 1], [0, 0, -1])
    assert out["flags"][0] == 0
