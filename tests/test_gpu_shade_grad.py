"""GPU shading gradient and the uniform estimator vs the oracle (Eq. 13-15).

The gradient holds the sample directions fixed on both sides; the oracle's
version is pinned by exact difference quotients (albedo, environment),
central differences (roughness under uniform sampling, surfels through the
traced rays) and an unbiasedness check against quadrature (roughness under
GGX sampling). Points whose traced rays carry an ambiguity flag get a zero
upstream gradient on both sides, so they contribute nothing. The ray-interval
margin is 2e-8 here instead of the default 1e-6: secondary rays start on the
surface, so many hits lie within 1e-6 of t_min = 1e-3, while the kernel's
depth pair near the origin is accurate to ~1e-9.

Bars (FP32 kernel vs FP64 oracle): per output tensor ||g - g_ref|| /
||g_ref|| <= 1e-3 and every element within 2e-3 max|g_ref|; per point
albedo / roughness gradients within 1e-3 max(1, |ref|) relative."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_15867_gb300 as irgs  # noqa: E402
from tests.gpu_util import dev, make_scene  # noqa: E402

SURFEL = ("means", "quats", "scales", "opacity", "features")
GRAD_MARGINS = oracle.Margins(t_abs=2e-8)


def opar(p):
    return oracle.Params(alpha_min=p.alpha_min, alpha_max=p.alpha_max, T_min=p.T_min, t_min=p.t_min,
                         t_max=p.t_max, feat_offset=p.feat_offset, feat_count=p.feat_count)


def omode(mode):
    return oracle.MODE_UNIFORM if mode == "uniform" else oracle.MODE_SPLIT


def rel_check(a, b, name, norm_tol=1e-3, el_tol=2e-3):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    if nb == 0:
        assert np.abs(a).max(initial=0.0) == 0.0, name
        return 0.0, 0.0
    rel = np.linalg.norm(a - b) / nb
    el = np.abs(a - b).max() / np.abs(b).max()
    assert rel <= norm_tol and el <= el_tol, (name, rel, el)
    return rel, el


def grads_both(sc, gb, env, nd, ns, seed, p, mode, flags_seed=11):
    x, n, a, r, wo = gb
    f = oracle.shade(sc, x, n, a, r, wo, env, nd, ns, seed, opar(p), margins=GRAD_MARGINS, mode=omode(mode))
    keep = f["flags"] == 0
    assert keep.mean() > 0.7, keep.mean()
    g = np.random.default_rng(flags_seed).normal(size=(x.shape[0], 3)).astype(np.float32)
    g[~keep] = 0.0
    S = make_scene(irgs, sc)
    out = irgs.shade_mc_backward(S, dev(x), dev(n), dev(a), dev(r), dev(wo), dev(env), nd, ns, seed, p, dev(g),
                                 mode=mode)
    torch.cuda.synchronize()
    assert S.status() == 0
    ref = oracle.shade_grad(sc, x, n, a, r, wo, env, nd, ns, seed, opar(p), g, mode=omode(mode))
    return {k: v.detach().cpu().numpy() for k, v in out.items()}, ref, keep


@pytest.mark.parametrize("mode,nd,ns,k,flags", [("split", 24, 24, 16, 0), ("uniform", 40, 0, 16, 0),
                                                ("split", 9, 7, 8, 0), ("split", 24, 24, 16, 1)])
def test_shading_gradient_matches_oracle(mode, nd, ns, k, flags):
    sc = synth.object_scene(n=8_000, seed=201)
    gb = synth.gbuffer_points(48, seed=202)
    env = synth.env_map(seed=203, height=32, width=64)
    p = irgs.TraceParams(k=k, feat_count=3, t_min=1e-3, flags=flags)
    got, ref, keep = grads_both(sc, gb, env, nd, ns, 77, p, mode)
    worst = {}
    for name in SURFEL + ("env",):
        b = ref[name] if name != "features" else ref[name][:, :3]
        a = got[name] if name != "features" else got[name][:, :3]
        worst[name] = rel_check(a, b, name)
    for name in ("albedo", "rough"):
        a, b = got[name][keep], ref[name][keep]
        err = np.abs(a - b).reshape(a.shape[0], -1).max(1) / np.maximum(
            1.0, np.abs(b).reshape(b.shape[0], -1).max(1))
        assert err.max() <= 1e-3, (name, err.max())
        worst[name] = float(err.max())
    print(worst)


def test_shading_gradient_traversal_modes_agree():
    sc = synth.object_scene(n=6_000, seed=211)
    x, n, a, r, wo = synth.gbuffer_points(40, seed=212)
    env = synth.env_map(seed=213, height=32, width=64)
    S = make_scene(irgs, sc)
    g = torch.from_numpy(np.random.default_rng(5).normal(size=(40, 3)).astype(np.float32)).cuda()
    p = irgs.TraceParams(k=16, feat_count=3, t_min=1e-3)
    args = (dev(x), dev(n), dev(a), dev(r), dev(wo), dev(env), 17, 15, 3)
    g1 = irgs.shade_mc_backward(S, *args, p, g)
    for fl in (irgs.FLAG_WARP, irgs.FLAG_PER_THREAD):
        g2 = irgs.shade_mc_backward(S, *args, p.with_(flags=fl), g)
        torch.cuda.synchronize()
        # same traces and per-sample arithmetic; atomics reorder the sums
        for k in g1:
            scale = max(float(g1[k].abs().max()), 1e-30)
            assert float((g1[k] - g2[k]).abs().max()) <= 1e-5 * scale, (fl, k)


def test_zero_upstream_gradient_adds_nothing():
    sc = synth.object_scene(n=3_000, seed=221)
    x, n, a, r, wo = synth.gbuffer_points(16, seed=222)
    env = synth.env_map(seed=223, height=16, width=32)
    S = make_scene(irgs, sc)
    p = irgs.TraceParams(k=8, feat_count=3, t_min=1e-3)
    out = irgs.shade_mc_backward(S, dev(x), dev(n), dev(a), dev(r), dev(wo), dev(env), 8, 8, 1, p,
                                 torch.zeros((16, 3), device="cuda"))
    torch.cuda.synchronize()
    for k, v in out.items():
        assert float(v.abs().max()) == 0.0, k


def test_autograd_shade_matches_direct_call():
    sc = synth.object_scene(n=4_000, seed=231)
    x, n, a, r, wo = synth.gbuffer_points(24, seed=232)
    env = synth.env_map(seed=233, height=16, width=32)
    p = irgs.TraceParams(k=16, feat_count=3, t_min=1e-3)
    leaves = [torch.tensor(v, device="cuda", requires_grad=True)
              for v in (sc.means, sc.quats, sc.scales, sc.opacity, sc.features)]
    S = irgs.Scene(*leaves, alpha_min=p.alpha_min)
    at = torch.tensor(a, device="cuda", requires_grad=True)
    rt = torch.tensor(r, device="cuda", requires_grad=True)
    et = torch.tensor(env, device="cuda", requires_grad=True)
    rgb = irgs.shade(S, dev(x), dev(n), at, rt, dev(wo), et, 12, 12, 4, p)
    ref = irgs.shade_mc(S, dev(x), dev(n), dev(a), dev(r), dev(wo), dev(env), 12, 12, 4, p)["rgb"]
    assert torch.equal(rgb.detach(), ref)
    g = torch.from_numpy(np.random.default_rng(7).normal(size=(24, 3)).astype(np.float32)).cuda()
    (rgb * g).sum().backward()
    direct = irgs.shade_mc_backward(S, dev(x), dev(n), dev(a), dev(r), dev(wo), dev(env), 12, 12, 4, p, g)
    torch.cuda.synchronize()
    pairs = list(zip(SURFEL, leaves)) + [("albedo", at), ("rough", rt), ("env", et)]
    for name, t in pairs:
        d = direct[name].reshape(t.shape)
        scale = max(float(d.abs().max()), 1e-30)
        assert float((t.grad - d).abs().max()) <= 1e-5 * scale, name


def check_fwd(out, ref, frac=0.999):
    gg = out["rgb"].cpu().numpy().astype(np.float64)
    err = np.abs(gg - ref["rgb"]).max(1) / np.maximum(1.0, np.abs(ref["rgb"]).max(1))
    ok = ref["flags"] == 0
    assert (err <= 1e-4).mean() >= frac, (err.max(), (err <= 1e-4).mean())
    assert np.all(err[ok] <= 2e-3), err[ok].max()
    for k in ("vis", "ind"):
        a = out[k].cpu().numpy().reshape(len(ok), -1)
        b = ref[k].reshape(len(ok), -1)
        assert np.all(np.abs(a - b).max(1)[ok] <= 1e-4 * np.maximum(1, np.abs(b).max(1)[ok])), k


@pytest.mark.parametrize("nd,k", [(48, 16), (5, 8), (33, 16)])
def test_uniform_estimator_matches_oracle(nd, k):
    sc = synth.object_scene(n=20_000, seed=241)
    gb = synth.gbuffer_points(64, seed=242)
    env = synth.env_map(seed=243, height=64, width=128)
    p = irgs.TraceParams(k=k, feat_count=3, t_min=1e-3)
    S = make_scene(irgs, sc)
    out = irgs.shade_mc(S, *(dev(v) for v in gb), dev(env), nd, 0, 55, p, want_aux=True, mode="uniform")
    torch.cuda.synchronize()
    assert S.status() == 0
    ref = oracle.shade(sc, *gb, env, nd, 0, 55, opar(p), mode=oracle.MODE_UNIFORM)
    check_fwd(out, ref, frac=0.98)


def test_uniform_mode_rejects_specular_samples():
    sc = synth.object_scene(n=1_000, seed=251)
    x, n, a, r, wo = synth.gbuffer_points(4, seed=252)
    env = synth.env_map(seed=253, height=8, width=16)
    S = make_scene(irgs, sc)
    p = irgs.TraceParams(k=8, feat_count=3, t_min=1e-3)
    with pytest.raises(irgs.IrgsError):
        irgs.shade_mc(S, dev(x), dev(n), dev(a), dev(r), dev(wo), dev(env), 4, 4, 0, p, mode="uniform")
    with pytest.raises(irgs.IrgsError):
        irgs.trace_forward(S, dev(x), dev(n), p.with_(flags=irgs.FLAG_UNIFORM))


def _faint_layers(layers=40, per=60, seed=221):
    """Horizontal layers of faint surfels above z = 0 (normal +z): secondary
    rays leaving the floor cross them all and blend ~100 hits each."""
    rng = np.random.default_rng(seed)
    n = layers * per
    means = np.column_stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n),
                             0.05 + 0.02 * np.repeat(np.arange(layers), per) + rng.uniform(0, 0.005, n)])
    quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    scales = np.exp(rng.normal(np.log(0.1), 0.2, size=(n, 2)))
    opacity = rng.uniform(0.02, 0.08, n)
    feats = rng.uniform(0, 1, (n, 3))
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return synth.Surfels(f(means), f(quats), f(scales), f(opacity), f(feats))


def test_wavefront_gradient_replays_rays_beyond_saved_lists():
    """The wavefront gradient saves 64 hit ids per secondary ray; rays that
    blend more replay their march from a list the listing launch builds.
    Here most rays do; the gradient must equal the fused per-thread kernel's
    (which replays every ray) up to the reordering of the float atomics."""
    sc = _faint_layers()
    P, nd, ns = 24, 16, 16
    rng = np.random.default_rng(222)
    x = np.column_stack([rng.uniform(-0.5, 0.5, P), rng.uniform(-0.5, 0.5, P), np.zeros(P)]).astype(np.float32)
    n = np.tile(np.float32([0, 0, 1]), (P, 1))
    a = rng.uniform(0.1, 0.9, (P, 3)).astype(np.float32)
    r = rng.uniform(0.2, 1.0, P).astype(np.float32)
    wo = n.copy()
    env = synth.env_map(seed=223, height=32, width=64)
    S = make_scene(irgs, sc)
    p = irgs.TraceParams(k=16, feat_count=3, t_min=1e-3)
    # the sampled rays really exceed the saved list length
    d, v = irgs.shade_sample_rays(dev(n), dev(r), dev(wo), nd, ns, 31)
    vm = v.bool()
    o = dev(x).repeat_interleave(nd + ns, 0)[vm].contiguous()
    nh = irgs.trace_forward(S, o, d[vm].contiguous(), p)["n_hits"].cpu().numpy()
    assert (nh > 64).sum() >= 50, np.sort(nh)[-10:]
    g = torch.from_numpy(rng.normal(size=(P, 3)).astype(np.float32)).cuda()
    args = (dev(x), dev(n), dev(a), dev(r), dev(wo), dev(env), nd, ns, 31)
    g1 = irgs.shade_mc_backward(S, *args, p, g)
    g2 = irgs.shade_mc_backward(S, *args, p.with_(flags=irgs.FLAG_PER_THREAD), g)
    torch.cuda.synchronize()
    assert S.status() == 0
    for k in g1:
        scale = max(float(g1[k].abs().max()), 1e-30)
        assert float((g1[k] - g2[k]).abs().max()) <= 1e-5 * scale, k
    assert float(g1["opacity"].abs().sum()) > 0
