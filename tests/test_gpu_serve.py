"""Serving path: persistent multi-request launches over resident scenes.

Each request's result must be the same whether it runs alone or in a mix
(bitwise: the per-ray and per-point computations do not depend on what
shares the launch), the serving kernel must agree with the standalone entry
points on the same rays / G-buffer, and served results are compared element
by element with the FP64 oracle on host-made rays and G-buffers."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_15867_gb300 as irgs  # noqa: E402
from paper_2412_15867_gb300 import serve  # noqa: E402
from tests.gpu_util import assert_forward_parity, dev, make_scene, oracle_reference  # noqa: E402

SCENE_ARGS = [(20_000, 401), (50_000, 402)]
ENV_ARGS = dict(seed=403, height=64, width=128)


@pytest.fixture(scope="module")
def scenes():
    return [make_scene(irgs, synth.object_scene(n=n, seed=s)) for n, s in SCENE_ARGS]


@pytest.fixture(scope="module")
def env():
    return dev(synth.env_map(**ENV_ARGS))


@pytest.mark.parametrize("tile", [(4, 8), (8, 4), (1, 1)])
def test_camera_rays_match_the_pinhole_model(tile):
    cam = serve.make_camera((3.0, -1.0, 2.0), 64, 32, fov_deg=50.0, tile=tile)
    o, d = serve.camera_rays(cam)
    ro, rd = synth.look_at_rays((3.0, -1.0, 2.0), (0, 0, 0), 64, 32, fov_deg=50.0, tile=tile)
    np.testing.assert_allclose(d.cpu().numpy(), rd, atol=3e-7)
    np.testing.assert_allclose(o.cpu().numpy(), ro, atol=0)


def test_render_equals_standalone_trace(scenes):
    S = scenes[0]
    srv = serve.Server([S], max_tiles=512)
    req = serve.RenderRequest(0, (3.5, 1.0, 2.0), 96, 64)
    h = srv.submit(req)
    srv.run_until_idle()
    o, d = serve.camera_rays(serve.make_camera(req.eye, req.width, req.height))
    ref = irgs.trace_forward(S, o, d, irgs.TraceParams(k=16, feat_count=10))
    torch.cuda.synchronize()
    for k in ("feat", "depth", "opacity"):
        assert torch.equal(h.out[k], ref[k]), k
    assert S.status() == 0
    srv.close()


def test_relight_equals_standalone_gbuffer_and_shading(scenes, env):
    S = scenes[1]
    srv = serve.Server([S], max_tiles=512)
    req = serve.RelightRequest(0, (-2.5, 2.5, 2.0), 64, 48, spp=12, env=env, seed=77)
    h = srv.submit(req)
    srv.run_until_idle()
    o, d = serve.camera_rays(serve.make_camera(req.eye, req.width, req.height))
    mat = irgs.trace_forward(S, o, d, irgs.TraceParams(k=16, feat_offset=3, feat_count=7))
    g = serve.gbuffer_views(h.out["gbuffer"], req.pixels())
    O = mat["opacity"]
    valid = O > 0.5
    assert torch.equal(g["valid"] > 0.5, valid)
    v = valid
    inv = 1.0 / O[v]
    torch.testing.assert_close(g["albedo"][v], mat["feat"][v, 0:3] * inv[:, None], rtol=1e-6, atol=1e-6)
    torch.testing.assert_close(g["rough"][v], mat["feat"][v, 3] * inv, rtol=1e-6, atol=1e-6)
    torch.testing.assert_close(g["x"][v], o[v] + d[v] * (mat["depth"][v] * inv)[:, None], rtol=1e-6, atol=1e-6)
    nn = mat["feat"][v, 4:7]
    torch.testing.assert_close(g["n"][v], nn / nn.norm(dim=1, keepdim=True), rtol=1e-5, atol=1e-6)
    torch.testing.assert_close(g["wo"][v], -d[v])
    # shading of the valid pixels with the standalone entry point: the same
    # wavefront path keyed by pixel index, so the estimates are identical
    ps = irgs.TraceParams(k=16, feat_count=3, t_min=1e-3)
    sh = irgs.shade_mc(S, g["x"], g["n"], g["albedo"], g["rough"], g["wo"], env, 6, 6, 77, ps)
    assert torch.equal(h.out["rgb"][v], sh["rgb"][v])
    assert torch.count_nonzero(h.out["rgb"][~v]) == 0
    assert v.float().mean() > 0.2
    srv.close()


def _mixed_requests(env):
    return [serve.RenderRequest(0, (3.0, 0.5, 2.0), 128, 128),
            serve.RelightRequest(1, (-3.0, 1.0, 2.5), 64, 64, spp=7, env=env, seed=5),
            serve.RenderRequest(1, (0.5, -3.5, 1.5), 256, 128),
            serve.RelightRequest(0, (2.0, 2.0, 3.0), 128, 64, spp=32, env=env, seed=6),
            serve.RelightRequest(1, (1.0, 3.0, 1.0), 32, 32, spp=1, env=env, seed=7),
            serve.RenderRequest(0, (-1.5, -3.0, 2.5), 64, 64)]


@pytest.mark.parametrize("use_graph", [True, False])
def test_each_result_is_the_same_alone_and_in_the_mix(scenes, env, use_graph):
    reqs = _mixed_requests(env)
    mix = serve.Server(scenes, max_tiles=1024, step_rays=1 << 18, use_graph=use_graph)
    hs = [mix.submit(r) for r in reqs]
    mix.run_until_idle()
    assert mix.steps > 2 and all(h.done > 0 for h in hs)
    for r, h in zip(reqs, hs):
        alone = serve.Server(scenes, max_tiles=1024, batching=False, use_graph=not use_graph)
        ha = alone.submit(r)
        alone.run_until_idle()
        for k in h.out:
            if k == "gbuffer":
                continue
            assert torch.equal(h.out[k], ha.out[k]), (type(r).__name__, k)
        alone.close()
    mix.close()


def test_admission_respects_the_memory_budget(scenes, env):
    reqs = _mixed_requests(env)
    budget = 1_600_000        # the largest request (256x128 render, 1.57 MB) fits alone
    srv = serve.Server(scenes, hbm_budget=budget, max_tiles=1024)
    hs = [srv.submit(r) for r in reqs]
    peak = 0
    while srv.step() or srv.waiting:
        peak = max(peak, srv.used)
        assert srv.used <= budget
    assert all(h.done > 0 for h in hs)
    assert srv.steps >= 3          # the budget forced requests to wait for each other
    srv.close()


def test_invalid_tile_table_is_rejected(scenes):
    srv = serve.Server(scenes[:1], max_tiles=16)
    t = srv.tiles_tab[0]
    t.kind, t.job, t.first, t.count = 0, 3, 0, 10    # job 3 of 0 jobs
    with pytest.raises(irgs.IrgsError):
        irgs._lib.check(srv.L.irgs_server_step(srv._h, 0, 1, 0, None), "step")
    srv.close()


def test_poisson_driver_reports_latency(scenes, env):
    rng = np.random.default_rng(0)

    def make(i):
        if i % 2 == 0:
            return serve.RenderRequest(int(rng.integers(0, 2)), (3.0, 0.0, 2.0), 64, 64)
        return serve.RelightRequest(int(rng.integers(0, 2)), (0.0, 3.0, 2.0), 32, 32, spp=4, env=env, seed=i)

    srv = serve.Server(scenes, max_tiles=1024)
    hs, wall, rays = serve.run_poisson(srv, make, rate=200.0, duration=0.5, warmup=0.1)
    st = serve.latency_stats(hs)
    assert st["n"] > 20 and st["p99_ms"] >= st["p50_ms"] > 0 and rays > 0
    srv.close()


def opar(p):
    return oracle.Params(alpha_min=p.alpha_min, alpha_max=p.alpha_max, T_min=p.T_min, t_min=p.t_min,
                         t_max=p.t_max, feat_offset=p.feat_offset, feat_count=p.feat_count)


def test_served_mix_matches_the_oracle(scenes, env):
    """One served mix, every served result checked element by element
    against the FP64 oracle on the same host-made inputs:
      * two render requests on two scenes with their own rays (ragged counts,
        several tiles each): feat / depth / opacity per ray (Eq. 8) at the
        forward bars, flagged rays against their admissible outcomes;
      * a relight request whose G-buffer is traced from its own rays: the
        served G-buffer against the Eq. 9 normalisation of the oracle's
        material trace (x = o + (D/O) d, normal, albedo, roughness, w_o,
        valid = O > 0.5) on unflagged pixels;
      * a relight request that shades a host-made G-buffer: its radiance
        against oracle.shade with the request's seed and its pixel indices as
        the random keys (Eq. 13-15), at the shading bars;
    with camera-driven requests of both kinds sharing the launches."""
    sc_np = [synth.object_scene(n=n, seed=s) for n, s in SCENE_ARGS]
    env_np = synth.env_map(**ENV_ARGS)
    cams = synth.hemisphere_cameras(4, seed=411)
    r0 = synth.camera_batch_rays(cams[:1], 37, 29)                 # 1,073 rays
    r1 = synth.camera_batch_rays(cams[1:2], 41, 23)                # 943 rays
    rg = synth.camera_batch_rays(cams[2:3], 32, 25)                # 800 rays
    P_sh = 45
    x, n, a, r, wo = synth.gbuffer_points(P_sh, seed=412)
    gb = serve.pack_gbuffer(dev(x), dev(n), dev(a), dev(r), dev(wo))
    req = [serve.RenderRequest(0, (0, 0, 4), r0[0].shape[0], 1, rays=(dev(r0[0]), dev(r0[1]))),
           serve.RenderRequest(1, (0, 0, 4), r1[0].shape[0], 1, rays=(dev(r1[0]), dev(r1[1]))),
           serve.RelightRequest(1, (0, 0, 4), rg[0].shape[0], 1, spp=6, env=env, seed=91,
                                rays=(dev(rg[0]), dev(rg[1]))),
           serve.RelightRequest(0, (0, 0, 4), P_sh, 1, spp=10, env=env, seed=92, gbuffer=gb)]
    mix = _mixed_requests(env)
    srv = serve.Server(scenes, max_tiles=1024, step_rays=1 << 16, tile_px=512)
    hs = [srv.submit(q) for q in (mix[0], req[0], mix[1], req[1], req[2], mix[3], req[3], mix[2])]
    srv.run_until_idle()
    torch.cuda.synchronize()
    assert srv.steps > 2 and all(h.done > 0 for h in hs)
    assert all(S.status() == 0 for S in scenes)
    h0, h1, hg, hsh = hs[1], hs[3], hs[4], hs[6]
    # render requests
    for h, (ro, rd), sc in ((h0, r0, sc_np[0]), (h1, r1, sc_np[1])):
        ref = oracle_reference(sc, ro, rd, opar(srv.render_p))
        st = assert_forward_parity(h.out, ref, sc.features, max_flagged=0.05)
        print("render", st)
    # relight G-buffer from the request's rays
    ro, rd = rg
    mp = srv.render_p.with_(feat_offset=3, feat_count=7)
    ref = oracle.trace(sc_np[1], ro, rd, opar(mp))
    g = {k: t.cpu().numpy().astype(np.float64) for k, t in serve.gbuffer_views(hg.out["gbuffer"], ro.shape[0]).items()}
    O = ref["opacity"]
    ok = ((ref["flags"] & oracle.FORWARD_FLAGS) == 0) & (np.abs(O - 0.5) > 1e-3)
    assert ok.mean() > 0.95
    valid = O > 0.5
    np.testing.assert_array_equal(g["valid"][ok] > 0.5, valid[ok])
    v = ok & valid
    assert v.sum() > 100
    C = ref["feat"]
    xr = ro + rd * (ref["depth"] / np.where(valid, O, 1))[:, None]
    nr = C[:, 4:7] / np.linalg.norm(C[:, 4:7], axis=1, keepdims=True).clip(1e-30)
    np.testing.assert_allclose(g["x"][v], xr[v], rtol=0, atol=5e-4)
    np.testing.assert_allclose(g["albedo"][v], C[v, 0:3] / O[v, None], rtol=0, atol=3e-4)
    np.testing.assert_allclose(g["rough"][v], C[v, 3] / O[v], rtol=0, atol=3e-4)
    wide = v & (np.linalg.norm(C[:, 4:7], axis=1) > 0.1)
    np.testing.assert_allclose(g["n"][wide], nr[wide], rtol=0, atol=3e-3)
    np.testing.assert_allclose(g["wo"][v], -rd[v], rtol=0, atol=0)
    np.testing.assert_allclose(g["opacity"][v], O[v], rtol=0, atol=1e-4)
    # relight shading of the host-made G-buffer
    # secondary rays start on the surface, so many points have a hit within
    # 1e-6 of t_min; the kernel resolves depths near the origin to ~1e-9, so
    # the ray-interval margin here is 2e-8 (as in the shading-gradient tests)
    sref = oracle.shade(sc_np[0], x, n, a, r, wo, env_np, 5, 5, 92, opar(srv.shade_p),
                        margins=oracle.Margins(t_abs=2e-8))
    rgb = hsh.out["rgb"].cpu().numpy().astype(np.float64)
    err = np.abs(rgb - sref["rgb"]).max(1) / np.maximum(1.0, np.abs(sref["rgb"]).max(1))
    clean = sref["flags"] == 0
    assert clean.mean() > 0.5 and np.all(err[clean] <= 1e-4), (err, sref["flags"])
    assert (err <= 1e-4).mean() >= 0.9, err
    # flagged points: inside the range their samples' admissible outcomes allow
    fl = np.nonzero(~clean)[0]
    if fl.size:
        b = oracle.shade_bounds(sc_np[0], x[fl], n[fl], a[fl], r[fl], wo[fl], env_np, 5, 5, 92, opar(srv.shade_p),
                                margins=oracle.Margins(t_abs=2e-8), point_ids=fl)
        tol = 1e-4 * np.maximum(1.0, np.abs(sref["rgb"][fl]).max(1))[:, None]
        assert np.all((rgb[fl] >= b["lo"] - tol) & (rgb[fl] <= b["hi"] + tol)), (rgb[fl], b)
    srv.close()


def test_oldest_request_is_not_starved(scenes):
    """A large request keeps a share of every step while more small work
    arrives each step than the step budget holds (shortest remaining work
    first alone would give the large request nothing): it finishes within a
    bounded number of steps."""
    srv = serve.Server(scenes, max_tiles=1024, step_rays=1 << 16, tile_px=1024)
    big = srv.submit(serve.RenderRequest(0, (3.0, 0.5, 2.0), 512, 512))      # 262,144 rays: 4 steps' budget
    small = []
    for i in range(40):
        for _ in range(5):                                                   # 5 x 16,384 rays per step
            small.append(srv.submit(serve.RenderRequest(1, (0.5, -3.5, 1.5), 128, 128)))
        srv.step()
        if big.done > 0:
            break
    # a quarter of each step's budget goes to the oldest request: 16 steps at most
    assert big.done > 0 and srv.steps <= 16, srv.steps
    srv.run_until_idle()
    assert all(h.done > 0 for h in small)
    assert all(S.status() == 0 for S in scenes)
    srv.close()
