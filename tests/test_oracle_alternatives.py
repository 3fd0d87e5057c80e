"""Pins of the oracle's admissible outcomes for rays whose exact answer lies
within a margin of a discontinuity (oracle_trace_alternatives): each is
checked against closed-form blends of the constructed hits (Eq. 2, Eq. 8),
not against the oracle's own compositing routine."""
import math

import numpy as np
from scipy.spatial.transform import Rotation

import oracle
from oracle import Margins, Params
import synth
from tests.helpers import quat_wxyz, rays, scene

P0 = Params(alpha_min=1 / 255, alpha_max=0.99, T_min=1e-4, t_min=0.0, t_max=math.inf,
            feat_offset=0, feat_count=3)
Q = quat_wxyz(Rotation.identity())          # normal +z


def outcomes(sc, o, d, params=P0, margins=Margins()):
    ro, rd = rays(o, d)
    a = oracle.trace_alternatives(sc, ro, rd, params, margins)
    c = int(a["count"][0])
    return c, [(a["feat"][0, j], a["depth"][0, j], a["opacity"][0, j], int(a["n_hits"][0, j])) for j in range(max(c, 1))]


def blend(hits):
    """Closed-form front-to-back blend of [(alpha, f, tau)]."""
    C, D, T = np.zeros(3), 0.0, 1.0
    for a, f, t in hits:
        C += T * a * np.asarray(f, np.float64)
        D += T * a * t
        T *= 1 - a
    return C, D, 1 - T


def match(outs, C, D, O, nh, tol=1e-9):
    return any(np.abs(f - C).max() < tol and abs(d - D) < tol and abs(o - O) < tol and n == nh
               for f, d, o, n in outs)


def test_first_outcome_is_the_definition():
    sc = synth.object_scene(n=3000, seed=31)
    ro, rd = synth.camera_batch_rays(synth.hemisphere_cameras(2, seed=31), 24, 20)
    p = Params(feat_count=10)
    ref = oracle.trace(sc, ro, rd, p)
    alt = oracle.trace_alternatives(sc, ro, rd, p)
    assert np.all(alt["count"] != 0)
    np.testing.assert_array_equal(alt["feat"][:, 0], ref["feat"])
    np.testing.assert_array_equal(alt["depth"][:, 0], ref["depth"])
    np.testing.assert_array_equal(alt["n_hits"][:, 0], ref["n_hits"])
    # unflagged rays have exactly one outcome
    clean = (ref["flags"] & oracle.FORWARD_FLAGS) == 0
    assert np.all(alt["count"][clean] == 1)


def test_near_tie_gives_both_orders():
    # two parallel surfels 1e-9 apart in depth: within the tie margin
    f1, f2 = [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]
    sc = scene([[0, 0, 0], [0, 0, -1e-9]], [Q, Q], [[0.3, 0.3]] * 2, [0.6, 0.3], [f1, f2])
    a1, a2 = (float(x) for x in sc.opacity)
    t1, t2 = 3.0, 3.0 + float(np.float32(1e-9))
    c, outs = outcomes(sc, [0, 0, 3], [0, 0, -1])
    assert c == 2
    C, D, O = blend([(a1, f1, t1), (a2, f2, t2)])
    assert match(outs[:1], C, D, O, 2)
    C, D, O = blend([(a2, f2, t2), (a1, f1, t1)])
    assert match(outs, C, D, O, 2)
    # 1e-3 apart: one order only
    sc2 = scene([[0, 0, 0], [0, 0, -1e-3]], [Q, Q], [[0.3, 0.3]] * 2, [0.6, 0.3], [f1, f2])
    c, _ = outcomes(sc2, [0, 0, 3], [0, 0, -1])
    assert c == 1


def test_candidate_at_the_alpha_cutoff_in_or_out():
    # a ray through the surfel where o exp(-rho^2/2) = alpha_min (1 + 1e-5):
    # below o = 0.35 the cutoff lies inside 3 sigma (and is the support edge
    # of Eq. 5), so the candidate is in or out
    o = 0.3
    s = 0.2
    amin = 1 / 255
    rho = math.sqrt(2 * math.log(o / (amin * (1 + 1e-5))))
    assert rho < 3
    f1, f2 = [0.2, 0.4, 0.6], [1.0, 1.0, 1.0]
    # surfel 0 at the cutoff, surfel 1 behind it, hit at its centre
    sc = scene([[rho * s, 0, 0], [0, 0, -0.5]], [Q, Q], [[s, s], [0.3, 0.3]], [o, 0.5], [f1, f2])
    o32 = float(sc.opacity[0])
    x = float(np.float32(rho * s))
    r2 = ((x - 0.0) / float(sc.scales[0, 0])) ** 2
    a_cut = o32 * math.exp(-r2 / 2)
    assert abs(a_cut - amin) < 1e-6
    c, outs = outcomes(sc, [0, 0, 3], [0, 0, -1])
    assert c == 2
    a2 = float(sc.opacity[1])
    C, D, O = blend([(a_cut, f1, 3.0), (a2, f2, 3.5)])
    assert match(outs, C, D, O, 2)
    C, D, O = blend([(a2, f2, 3.5)])
    assert match(outs, C, D, O, 1)


def test_stop_near_the_threshold_on_either_side():
    # identical stacked surfels at alpha = 0.9: T after hit j is 0.1^j; with
    # T_min = 1e-3 (1 + 1e-6) the stop after hit 3 is within the margin
    n = 6
    mus = [[0, 0, -0.1 * i] for i in range(n)]
    feats = [[1.0 * i, 0, 0] for i in range(n)]
    sc = scene(mus, [Q] * n, [[0.3, 0.3]] * n, [0.9] * n, feats)
    a = float(sc.opacity[0])
    Tafter3 = (1 - a) ** 3
    p = Params(feat_count=3, T_min=Tafter3 * (1 + 1e-6))
    c, outs = outcomes(sc, [0, 0, 3], [0, 0, -1], params=p)
    assert c == 3
    hits = [(a, feats[i], 3.0 + 0.1 * i) for i in range(n)]
    for k in (3, 4):
        C, D, O = blend(hits[:k])
        assert match(outs, C, D, O, k, tol=1e-7)
    # far from the threshold: a single outcome
    c, _ = outcomes(sc, [0, 0, 3], [0, 0, -1], params=Params(feat_count=3, T_min=Tafter3 * 1.5))
    assert c == 1


def test_too_many_outcomes_left_unresolved():
    # 30 coincident copies: a run of 30 tied hits cannot be listed
    sc = scene([[0, 0, 0]] * 30, [Q] * 30, [[0.3, 0.3]] * 30, [0.2] * 30,
               np.random.default_rng(0).uniform(size=(30, 3)))
    c, outs = outcomes(sc, [0, 0, 3], [0, 0, -1], params=Params(feat_count=3, T_min=0.0))
    assert c == -1
    ref = oracle.trace(sc, *rays([0, 0, 3], [0, 0, -1]), Params(feat_count=3, T_min=0.0))
    np.testing.assert_array_equal(outs[0][0], ref["feat"][0])


def test_shade_bounds_equal_the_estimate_where_nothing_is_ambiguous():
    sc = synth.object_scene(n=3000, seed=33)
    gb = synth.gbuffer_points(24, seed=34)
    env = synth.env_map(seed=35, height=16, width=32)
    p = Params(feat_count=3, t_min=1e-3)
    ref = oracle.shade(sc, *gb, env, 8, 8, 7, p)
    b = oracle.shade_bounds(sc, *gb, env, 8, 8, 7, p)
    assert np.all(b["lo"] <= ref["rgb"] + 1e-12) and np.all(ref["rgb"] <= b["hi"] + 1e-12)
    clean = ref["flags"] == 0
    assert clean.any()
    np.testing.assert_allclose(b["lo"][clean], ref["rgb"][clean], rtol=0, atol=1e-12)
    np.testing.assert_allclose(b["hi"][clean], ref["rgb"][clean], rtol=0, atol=1e-12)


def test_shade_bounds_span_both_orders_of_a_near_tie():
    # a point under two large parallel canopy disks 1e-9 apart in height:
    # every upward sample meets both at near-equal depths, so either order
    # is admissible; with f1 = red and f2 = green the two orders' indirect
    # light is (a1, (1 - a1) a2) or ((1 - a2) a1, a2) for the ray's alphas
    f1, f2 = [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]
    sc = scene([[0, 0, 1.0], [0, 0, 1.0 + 1e-9]], [Q, Q], [[10.0, 10.0]] * 2, [0.5, 0.7], [f1, f2])
    x = np.zeros((1, 3), np.float32)
    n = np.array([[0, 0, 1.0]], np.float32)
    alb = np.array([[0.5, 0.6, 0.7]], np.float32)
    rough = np.array([0.5], np.float32)
    L = np.array([1.5, 0.5, 0.25], np.float32)
    env = np.tile(L, (8, 16, 1)).astype(np.float32)
    p = Params(feat_count=3, t_min=1e-3)
    nd = 16
    b = oracle.shade_bounds(sc, x, n, alb, rough, n, env, nd, 0, 11, p)
    ref = oracle.shade(sc, x, n, alb, rough, n, env, nd, 0, 11, p)
    # the per-sample definitions from the oracle's own trace of the same directions
    dirs, valid = oracle.sample_dirs(n, n, rough, nd, 0, 11)
    d = dirs[0][valid[0]]
    tr = oracle.trace(sc, np.zeros_like(d, dtype=np.float32), d.astype(np.float32), p)
    a1 = tr["feat"][:, 0]
    a2 = tr["feat"][:, 1] / (1 - a1)
    V = 1 - tr["opacity"]
    assert np.all(a1 > 0.4) and np.all(a2 > 0.5)
    defn = np.stack([a1, (1 - a1) * a2, 0 * a1], 1)
    swap = np.stack([(1 - a2) * a1, a2, 0 * a1], 1)
    t_def = alb[0] * (V[:, None] * L + defn) / nd
    t_swp = alb[0] * (V[:, None] * L + swap) / nd
    # (the check trace takes the directions rounded to float32, the
    # estimate its FP64 directions: agreement to ~1e-9)
    np.testing.assert_allclose(ref["rgb"][0], t_def.sum(0), rtol=1e-7)
    np.testing.assert_allclose(b["lo"][0], np.minimum(t_def, t_swp).sum(0), rtol=1e-7)
    np.testing.assert_allclose(b["hi"][0], np.maximum(t_def, t_swp).sum(0), rtol=1e-7)
    assert b["hi"][0, 1] - b["lo"][0, 1] > 1e-3


def test_relight_bounds_equal_the_estimate_where_nothing_is_ambiguous():
    sc = synth.object_scene(n=3000, seed=36)
    x, n, a, r, wo = synth.gbuffer_points(16, seed=37)
    env = synth.env_map(seed=38, height=16, width=32)
    p = Params(feat_offset=3, feat_count=7, t_min=1e-3)
    ref = oracle.relight(sc, x, n, a, r, wo, env, 16, 5, p)
    b = oracle.relight_bounds(sc, x, n, a, r, wo, env, 16, 5, p)
    assert np.all(b["lo"] <= ref["rgb"] + 1e-12) and np.all(ref["rgb"] <= b["hi"] + 1e-12)
    clean = ref["flags"] == 0
    assert clean.any()
    np.testing.assert_allclose(b["lo"][clean], ref["rgb"][clean], rtol=0, atol=1e-12)
    np.testing.assert_allclose(b["hi"][clean], ref["rgb"][clean], rtol=0, atol=1e-12)


def test_relight_bounds_widen_under_a_near_tie():
    # two large canopy disks 1e-9 apart with different albedo and roughness
    # channels: the two blend orders give different traced materials, so the
    # range has width, and the definition's estimate lies inside it
    f1 = [0, 0, 0, 0.9, 0.1, 0.1, 0.2, 0, 0, 1]
    f2 = [0, 0, 0, 0.1, 0.8, 0.3, 0.9, 0, 0, 1]
    sc = scene([[0, 0, 1.0], [0, 0, 1.0 + 1e-9]], [Q, Q], [[10.0, 10.0]] * 2, [0.5, 0.7], [f1, f2])
    x = np.zeros((1, 3), np.float32)
    n = np.array([[0, 0, 1.0]], np.float32)
    alb = np.array([[0.5, 0.6, 0.7]], np.float32)
    rough = np.array([0.5], np.float32)
    env = synth.env_map(seed=39, height=16, width=32)
    p = Params(feat_offset=3, feat_count=7, t_min=1e-3)
    ref = oracle.relight(sc, x, n, alb, rough, n, env, 32, 3, p)
    b = oracle.relight_bounds(sc, x, n, alb, rough, n, env, 32, 3, p)
    assert ref["flags"][0] & oracle.F_TIE
    assert np.all(b["lo"][0] <= ref["rgb"][0] + 1e-12) and np.all(ref["rgb"][0] <= b["hi"][0] + 1e-12)
    assert (b["hi"][0] - b["lo"][0]).max() > 1e-4
