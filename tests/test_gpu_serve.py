"""Serving path: persistent multi-request launches over resident scenes.

Each request's result must be the same whether it runs alone or in a mix
(bitwise: the per-ray and per-point computations do not depend on what
shares the launch), and the serving kernel must agree with the standalone
entry points on the same rays / G-buffer (which are oracle-checked)."""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_15867_gb300 as irgs  # noqa: E402
from paper_2412_15867_gb300 import serve  # noqa: E402
from tests.gpu_util import dev, make_scene  # noqa: E402


@pytest.fixture(scope="module")
def scenes():
    a = make_scene(irgs, synth.object_scene(n=20_000, seed=401))
    b = make_scene(irgs, synth.object_scene(n=50_000, seed=402))
    return [a, b]


@pytest.fixture(scope="module")
def env():
    return dev(synth.env_map(seed=403, height=64, width=128))


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
    g = h.out["gbuffer"]
    O = mat["opacity"]
    valid = O > 0.5
    assert torch.equal(g[:, 13] > 0.5, valid)
    v = valid
    inv = 1.0 / O[v]
    torch.testing.assert_close(g[v, 6:9], mat["feat"][v, 0:3] * inv[:, None], rtol=1e-6, atol=1e-6)
    torch.testing.assert_close(g[v, 9], mat["feat"][v, 3] * inv, rtol=1e-6, atol=1e-6)
    torch.testing.assert_close(g[v, 0:3], o[v] + d[v] * (mat["depth"][v] * inv)[:, None], rtol=1e-6, atol=1e-6)
    nn = mat["feat"][v, 4:7]
    torch.testing.assert_close(g[v, 3:6], nn / nn.norm(dim=1, keepdim=True), rtol=1e-5, atol=1e-6)
    torch.testing.assert_close(g[v, 10:13], -d[v])
    # shading of the valid pixels with the standalone entry point
    ps = irgs.TraceParams(k=16, feat_count=3, t_min=1e-3)
    sh = irgs.shade_mc(S, g[:, 0:3], g[:, 3:6], g[:, 6:9], g[:, 9].contiguous(), g[:, 10:13].contiguous(), env,
                       6, 6, 77, ps)
    torch.testing.assert_close(h.out["rgb"][v], sh["rgb"][v], rtol=1e-6, atol=1e-6)
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
