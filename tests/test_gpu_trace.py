"""GPU forward trace vs the FP64 oracle (through the C ABI), LBVH structure
invariants, k-buffer independence and edge cases."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import synth
from tests.helpers import frame_of, quat_wxyz, rays, scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_15867_gb300 as irgs  # noqa: E402
from tests.gpu_util import assert_forward_parity, dev, forward_errors, make_scene, oracle_reference  # noqa: E402


def opar(p):
    return oracle.Params(alpha_min=p.alpha_min, alpha_max=p.alpha_max, T_min=p.T_min, t_min=p.t_min,
                         t_max=p.t_max, feat_offset=p.feat_offset, feat_count=p.feat_count)


def run(sc, ro, rd, p, ids=0):
    S = make_scene(irgs, sc)
    out = irgs.trace_forward(S, dev(ro), dev(rd), p, max_hit_ids=ids)
    torch.cuda.synchronize()
    assert S.status() == 0
    return S, out


def test_tiny_config_all_rays_match_oracle():
    # 1,024 surfels, 64x64 camera rays, k = 8, alpha cutoff 1/255, T_min 1e-4
    sc = synth.tiny_scene(seed=1000, n=1024)
    ro, rd = synth.look_at_rays(synth.tiny_camera(1000), (0, 0, 0), 64, 64)
    p = irgs.TraceParams(k=8, feat_count=3)
    _, out = run(sc, ro, rd, p, ids=64)
    ref = oracle_reference(sc, ro, rd, opar(p), max_ids=64)
    st = assert_forward_parity(out, ref, sc.features, check_ids=True, max_flagged=0.02)
    assert (out["n_hits"].cpu().numpy() > 0).mean() > 0.5
    print(st)


@pytest.mark.parametrize("n,cams,w,h", [(10_000, 3, 37, 53), (2_000, 2, 129, 7)])
def test_object_scene_ragged_batches(n, cams, w, h):
    sc = synth.object_scene(n=n, seed=1001)
    ro, rd = synth.camera_batch_rays(synth.hemisphere_cameras(cams, seed=1001), w, h)
    p = irgs.TraceParams(k=16, feat_offset=0, feat_count=10)
    _, out = run(sc, ro, rd, p, ids=32)
    ref = oracle_reference(sc, ro, rd, opar(p), max_ids=32)
    assert_forward_parity(out, ref, sc.features, check_ids=True)


def test_results_independent_of_k():
    sc = synth.object_scene(n=20_000, seed=5)
    ro, rd = synth.camera_batch_rays(synth.hemisphere_cameras(2, seed=5), 64, 48)
    S = make_scene(irgs, sc)
    outs = {}
    for k in (1, 4, 8, 16, 32):
        p = irgs.TraceParams(k=k, feat_count=10)
        outs[k] = irgs.trace_forward(S, dev(ro), dev(rd), p, max_hit_ids=24)
    base = outs[16]
    for k, o in outs.items():
        for key in ("feat", "depth", "opacity", "n_hits", "hit_ids"):
            assert torch.equal(o[key], base[key]), (k, key)


def test_feature_channel_ranges():
    sc = synth.object_scene(n=5_000, seed=9)
    ro, rd = synth.camera_batch_rays(synth.hemisphere_cameras(1, seed=9), 40, 40)
    S = make_scene(irgs, sc)
    for off, cnt in ((0, 3), (3, 4), (6, 1), (0, 10), (9, 1), (0, 0)):
        p = irgs.TraceParams(k=16, feat_offset=off, feat_count=cnt)
        out = irgs.trace_forward(S, dev(ro), dev(rd), p)
        ref = oracle_reference(sc, ro, rd, opar(p))
        assert_forward_parity(out, ref)


def test_closed_forms_on_gpu():
    # two parallel surfels sharing frame and scales, rays along the normal at
    # local offsets (a, b): alpha_i = o_i exp(-(a^2+b^2)/2), blended front to back
    q = quat_wxyz(Rotation.from_rotvec([0.4, 0.9, -0.2]))
    tu, tv, n = frame_of(q)
    mu = np.array([-0.4, 0.1, 0.2])
    sc = scene([mu, mu - 0.3 * n], [q, q], [[0.03, 0.11]] * 2, [0.8, 0.6], [[1, 0, 0], [0, 1, 0]])
    s32 = sc.scales[0].astype(np.float64)
    offs = ((0, 0), (0.7, -1.3), (-1.9, 0.4), (3.2, 0.0))
    pts = [mu + a * s32[0] * tu + b * s32[1] * tv for a, b in offs]
    ro, rd = rays([p + 1.7 * n for p in pts], [-n] * len(pts))
    p = irgs.TraceParams(k=8, feat_count=3)
    _, out = run(sc, ro, rd, p)
    o1, o2 = float(sc.opacity[0]), float(sc.opacity[1])
    for i, (a, b) in enumerate(offs[:3]):
        G = math.exp(-(a * a + b * b) / 2)
        a1, a2 = o1 * G, o2 * G
        assert out["n_hits"][i].item() == 2
        np.testing.assert_allclose(out["feat"][i, 0].item(), a1, rtol=3e-6, atol=1e-7)
        np.testing.assert_allclose(out["feat"][i, 1].item(), (1 - a1) * a2, rtol=3e-6, atol=1e-7)
        np.testing.assert_allclose(out["opacity"][i].item(), 1 - (1 - a1) * (1 - a2), rtol=3e-6, atol=1e-7)
        np.testing.assert_allclose(out["depth"][i].item(), a1 * 1.7 + (1 - a1) * a2 * 2.0, rtol=3e-6)
    # beyond the 3-sigma support: no hit
    assert out["n_hits"][3].item() == 0


def test_edge_cases_empty_single_and_duplicates():
    p = irgs.TraceParams(k=8, feat_count=3)
    ro, rd = synth.look_at_rays(synth.tiny_camera(3), (0, 0, 0), 16, 16)
    # empty scene
    empty = scene(np.zeros((0, 3)), np.zeros((0, 4)), np.zeros((0, 2)), np.zeros(0), np.zeros((0, 3)))
    _, out = run(empty, ro, rd, p)
    assert torch.count_nonzero(out["opacity"]) == 0 and torch.count_nonzero(out["n_hits"]) == 0
    # one large surfel facing the camera
    cam = synth.tiny_camera(3)
    nrm = cam / np.linalg.norm(cam)
    from synth import frame_to_quat
    t_u = np.cross([0, 0, 1.0], nrm); t_u /= np.linalg.norm(t_u)
    t_v = np.cross(nrm, t_u)
    q = frame_to_quat(t_u[None], t_v[None], nrm[None])[0]
    one = scene([0, 0, 0], q, [0.3, 0.2], [0.9], [0.5, 0.25, 1.0])
    _, out = run(one, ro, rd, p)
    ref = oracle_reference(one, ro, rd, opar(p))
    assert_forward_parity(out, ref)
    assert out["n_hits"].sum().item() > 10
    # many exact duplicates (equal Morton codes, equal depths: ties by user index)
    base = synth.tiny_scene(seed=4, n=8)
    idx = np.repeat(np.arange(8), 40)
    dup = base.subset(idx)
    dup.features[:] = np.random.default_rng(0).uniform(0, 1, size=dup.features.shape).astype(np.float32)
    dup.scales[:] *= 4
    _, out = run(dup, ro, rd, p.with_(T_min=0.0), ids=64)
    ref = oracle_reference(dup, ro, rd, opar(p.with_(T_min=0.0)), max_ids=64)
    # runs of 40 tied hits are too many orders to list (unresolved), but
    # copies have bitwise-equal records, so their keys tie exactly on the GPU
    # as in FP64 and the user index decides: on rays whose only near-equal
    # depths are between copies of one surfel, the result is the definition's
    assert_forward_parity(out, ref, max_unresolved=1.0)
    tau, ids = ref["tau"], ref["ids"]
    near = np.abs(np.diff(tau, axis=1)) < 1e-6
    same = (ids[:, 1:] // 40) == (ids[:, :-1] // 40)
    only_copies = ~np.any(near & ~same & (ids[:, 1:] >= 0), axis=1)
    assert only_copies.mean() > 0.9
    err = forward_errors(out, ref)
    assert np.all(err[only_copies] <= 1e-4), err[only_copies].max()
    gid = out["hit_ids"].cpu().numpy()
    assert np.array_equal(gid[only_copies], ids[only_copies])
    assert (out["n_hits"].cpu().numpy()[only_copies] > 40).any()
    # zero rays
    S = make_scene(irgs, base)
    z = torch.zeros((0, 3), device="cuda:0")
    out = irgs.trace_forward(S, z, z, p)
    assert out["feat"].shape == (0, 3)


def test_ray_interval_and_parameter_validation():
    sc = synth.tiny_scene(seed=12, n=512)
    ro, rd = synth.random_rays_through_scene(2000, seed=13)
    S = make_scene(irgs, sc)
    for p in (irgs.TraceParams(k=8, t_min=2.5), irgs.TraceParams(k=16, t_min=1.0, t_max=3.0),
              irgs.TraceParams(k=8, alpha_max=1.0, T_min=0.0), irgs.TraceParams(k=8, alpha_min=0.05)):
        out = irgs.trace_forward(S, dev(ro), dev(rd), p)
        ref = oracle_reference(sc, ro, rd, opar(p))
        assert_forward_parity(out, ref)
    with pytest.raises(irgs.IrgsError):
        irgs.trace_forward(S, dev(ro), dev(rd), irgs.TraceParams(k=7))
    with pytest.raises(irgs.IrgsError):
        irgs.trace_forward(S, dev(ro), dev(rd), irgs.TraceParams(alpha_min=1e-4))   # below the scene's cutoff
    with pytest.raises(irgs.IrgsError):
        irgs.trace_forward(S, dev(ro), dev(rd), irgs.TraceParams(feat_offset=2, feat_count=3))
    with pytest.raises(irgs.IrgsError):
        irgs.trace_forward(S, dev(ro), dev(rd), irgs.TraceParams(t_min=-1.0))


def test_lbvh_structure_invariants():
    sc = synth.object_scene(n=30_000, seed=21)
    # add exact duplicates so equal Morton codes occur
    sc = sc.subset(np.concatenate([np.arange(sc.n), np.arange(500)]))
    S = make_scene(irgs, sc)
    perm, keys, nodes, boxes = S.export()
    n = sc.n
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.all(np.diff(keys.astype(np.int64)) >= 0)
    eq = np.diff(keys.astype(np.int64)) == 0
    assert np.all(np.diff(perm)[eq] > 0), "sort is not stable"
    ch = nodes[:, 12:14].view(np.int32)
    seen_leaf = np.zeros(n, np.int32)
    seen_node = np.zeros(n - 1, np.int32)
    stack = [0]
    seen_node[0] = 1
    while stack:
        i = stack.pop()
        b = [nodes[i, 0:6], np.r_[nodes[i, 6:9], nodes[i, 9:12]]]
        for s, c in enumerate(ch[i]):
            lo, hi = b[s][:3], b[s][3:]
            if c < 0:
                seen_leaf[~c] += 1
                assert np.all(lo <= boxes[~c, :3]) and np.all(hi >= boxes[~c, 3:])
            else:
                seen_node[c] += 1
                cb = np.r_[np.minimum(nodes[c, 0:3], nodes[c, 6:9]), np.maximum(nodes[c, 3:6], nodes[c, 9:12])]
                assert np.all(lo <= cb[:3]) and np.all(hi >= cb[3:])
                stack.append(c)
    assert np.all(seen_leaf == 1) and np.all(seen_node == 1)
    # leaf boxes contain the support ellipse (sampled on its rim)
    rng = np.random.default_rng(0)
    m = rng.integers(0, n, size=300)
    for mm in m:
        u = perm[mm]
        q = sc.quats[u].astype(np.float64)
        tu, tv, nrm = frame_of(q / np.linalg.norm(q))
        rc = min(3.0, math.sqrt(2 * math.log(float(sc.opacity[u]) * 255.0))) if sc.opacity[u] > 1 / 255 else 0.0
        th = np.linspace(0, 2 * math.pi, 64)
        pts = sc.means[u] + rc * (np.outer(np.cos(th), sc.scales[u, 0] * tu) + np.outer(np.sin(th), sc.scales[u, 1] * tv))
        assert np.all(pts >= boxes[mm, :3] - 1e-7) and np.all(pts <= boxes[mm, 3:] + 1e-7)


@pytest.mark.slow
def test_camera_config_full_size_sampled():
    """300k-surfel object scene, 100 cameras x 800x800 = 64M rays in 4x8 pixel
    tiles, k = 16, 10 channels, warp-coherent traversal with 96 saved hit ids:
    the full batch in the benchmark's launch configuration. Checked against
    the oracle element by element on 2,048 random rays, the 256 rays with the
    most blended hits and 256 rays that need four or more k-buffer rounds
    (the compacted rounds' run-to-completion launch); invariants on all rays.
    Flagged rays are checked against their admissible outcomes; at most 5%
    of the random sample may carry a flag (measured: ~3%, nearly all of them
    near-equal depths of nearly coplanar surfels 2e-8..7e-8 apart, under the
    2e-8 max(1, tau) tie margin)."""
    sc = synth.object_scene(n=300_000, seed=1001)
    cams = synth.hemisphere_cameras(100, seed=1001)
    ro, rd = synth.camera_batch_rays(cams, 800, 800, tile=(4, 8))
    p = irgs.TraceParams(k=16, feat_count=10)
    S = make_scene(irgs, sc)
    out = irgs.trace_forward(S, dev(ro), dev(rd), p, max_hit_ids=96)
    torch.cuda.synchronize()
    assert S.status() == 0
    o = out["opacity"]
    assert torch.isfinite(out["feat"]).all() and (o >= 0).all() and (o <= 1).all()
    nh_all = out["n_hits"]
    rng = np.random.default_rng(7)
    rand = rng.choice(ro.shape[0], 2048, replace=False)
    top = torch.topk(nh_all, 256).indices.cpu().numpy()
    deep = torch.nonzero(nh_all > 48).flatten().cpu().numpy()
    assert deep.size > 256
    deep = rng.choice(deep, 256, replace=False)
    for name, idx in (("random", rand), ("most hits", top), ("4+ rounds", deep)):
        idx = np.unique(idx)
        ref = oracle_reference(sc, ro[idx], rd[idx], opar(p), max_ids=96)
        ti = torch.from_numpy(idx).cuda()
        sub = {k: v[ti] for k, v in out.items()}
        st = assert_forward_parity(sub, ref, sc.features, check_ids=True,
                                   max_flagged=0.05 if name == "random" else 0.15)
        print(name, st, "mean hits", float(sub["n_hits"].float().mean()))


def test_traversal_modes_give_identical_results():
    """Warp-coherent and per-ray traversal return bit-identical outputs
    (the k-buffer holds the K nearest hits whatever the visiting order)."""
    sc = synth.object_scene(n=20_000, seed=15)
    ro, rd = synth.camera_batch_rays(synth.hemisphere_cameras(2, seed=15), 61, 33)
    ri, di = synth.random_rays_through_scene(3000, seed=16, box=2.0, radius=4.0)
    S = make_scene(irgs, sc)
    for o, d in ((ro, rd), (ri, di)):
        for k in (4, 8, 16, 32):
            pw = irgs.TraceParams(k=k, feat_count=10)
            a = irgs.trace_forward(S, dev(o), dev(d), pw, max_hit_ids=16)
            for fl in (irgs.FLAG_PER_THREAD, irgs.FLAG_WARP):
                b = irgs.trace_forward(S, dev(o), dev(d), pw.with_(flags=fl), max_hit_ids=16)
                for key in a:
                    assert torch.equal(a[key], b[key]), (k, fl, key)
    with pytest.raises(irgs.IrgsError):
        irgs.trace_forward(S, dev(ro), dev(rd), irgs.TraceParams(flags=3))
    with pytest.raises(irgs.IrgsError):
        irgs.trace_forward(S, dev(ro), dev(rd), irgs.TraceParams(flags=4))


def test_compacted_rounds_equal_per_ray_march():
    """Batches of 2^20 rays or more take the compacted rounds (rays still
    marching after round 1, 2 and 3 are regrouped into full warps; the rest
    run to completion): every output, the hit lists included, equals the
    per-ray march bit for bit, also for rays that need 4 rounds or more."""
    sc = synth.object_scene(n=300_000, seed=1001)
    ro, rd = synth.camera_batch_rays(synth.hemisphere_cameras(2, seed=17), 800, 700, tile=(4, 8))
    assert ro.shape[0] >= 1 << 20
    S = make_scene(irgs, sc)
    pw = irgs.TraceParams(k=16, feat_count=10)
    a = irgs.trace_forward(S, dev(ro), dev(rd), pw, max_hit_ids=96)
    b = irgs.trace_forward(S, dev(ro), dev(rd), pw.with_(flags=irgs.FLAG_PER_THREAD), max_hit_ids=96)
    torch.cuda.synchronize()
    assert S.status() == 0
    nh = a["n_hits"].cpu().numpy()
    assert (nh > 48).any() and (nh > 16).mean() > 0.3     # rounds 4+ (run to completion) and the compacted rounds both occur
    for key in a:
        assert torch.equal(a[key], b[key]), key


def test_trace_stats_counters_are_consistent():
    sc = synth.object_scene(n=20_000, seed=17)
    ro, rd = synth.camera_batch_rays(synth.hemisphere_cameras(1, seed=17), 64, 64, tile=(8, 4))
    S = make_scene(irgs, sc)
    p = irgs.TraceParams(k=16, feat_count=10)
    out = irgs.trace_forward(S, dev(ro), dev(rd), p)
    nh = out["n_hits"].cpu().numpy()
    sw = irgs.trace_stats(S, dev(ro), dev(rd), p).cpu().numpy()
    st = irgs.trace_stats(S, dev(ro), dev(rd), p.with_(flags=irgs.FLAG_PER_THREAD)).cpu().numpy()
    for s in (sw, st):
        assert np.array_equal(s[:, 0], sw[:, 0])          # rounds depend only on the hits
        assert np.all(s[:, 0] >= 1)
        assert np.all(s[:, 0] >= np.ceil(nh / 16))
        assert np.all(s[:, 3] >= nh) and np.all(s[:, 2] >= s[:, 3])
        assert np.all(s[nh > 0, 1] > 0)


def test_wide_hierarchy_invariants():
    sc = synth.object_scene(n=30_000, seed=23)
    sc = sc.subset(np.concatenate([np.arange(sc.n), np.arange(300)]))
    S = make_scene(irgs, sc)
    perm, keys, nodes, boxes = S.export()
    W = S.export_wide()
    n = sc.n
    assert 1 <= W.shape[0] <= n - 1          # each wide node takes at least one binary internal node
    lo = W[:, 0:12].reshape(-1, 3, 4)       # [node, axis, child]
    hi = W[:, 12:24].reshape(-1, 3, 4)
    ch = W[:, 24:28].view(np.int32)
    cnt = W[:, 28:29].view(np.int32)[:, 0]
    seen_leaf = np.zeros(n, np.int32)
    seen = np.zeros(W.shape[0], np.int32)
    seen[0] = 1
    stack = [0]
    while stack:
        w = stack.pop()
        valid = ch[w] != np.iinfo(np.int32).min
        assert valid.sum() == cnt[w] and 2 <= cnt[w] <= 4
        for k in np.nonzero(valid)[0]:
            c = ch[w, k]
            if c < 0:
                seen_leaf[~c] += 1
                assert np.array_equal(lo[w, :, k], boxes[~c, :3]) and np.array_equal(hi[w, :, k], boxes[~c, 3:])
            else:
                seen[c] += 1
                cv = ch[c] != np.iinfo(np.int32).min
                assert np.all(lo[w, :, k][:, None] <= lo[c][:, cv]) and np.all(hi[w, :, k][:, None] >= hi[c][:, cv])
                stack.append(c)
    assert np.all(seen_leaf == 1) and np.all(seen == 1)
