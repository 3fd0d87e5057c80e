"""Full-size checks in the benchmark's launch configurations for the paths
whose oracle comparisons otherwise run on small scenes: the camera backward
(64M rays, listed from 96 saved hit ids), the Monte Carlo shading gradient
(1M surfels, 640k points x 64 samples) and relighting (640k points x 64
environment samples); and the wavefront's chunking (at most 2^26 rays per
chunk, whole points) on a batch that spans two chunks.

A gradient summed over every ray is beyond the oracle at this size, so the
checks are (a) element by element against the oracle on sampled rays or
points, run through the same entry points with the full-size inputs (the
saved hit lists of the full forward, the points' own random keys), and (b)
linearity: the gradient of the whole batch equals the sum over chunks of it
(within the reordering of the float atomics)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import paper_2412_15867_gb300 as irgs  # noqa: E402
from tests.gpu_util import dev, make_scene  # noqa: E402

NAMES = ("means", "quats", "scales", "opacity", "features")
GRAD_FLAGS = oracle.FORWARD_FLAGS | oracle.F_CLAMP


def opar(p):
    return oracle.Params(alpha_min=p.alpha_min, alpha_max=p.alpha_max, T_min=p.T_min, t_min=p.t_min,
                         t_max=p.t_max, feat_offset=p.feat_offset, feat_count=p.feat_count)


def test_camera_backward_full_size():
    sc = synth.object_scene(n=300_000, seed=1001)
    cams = synth.hemisphere_cameras(100, seed=1001)
    ro, rd = synth.camera_batch_rays(cams, 800, 800, tile=(4, 8))
    R, F = ro.shape[0], 10
    gf, gd, go = synth.upstream_grads(R, F, seed=1004)
    S = make_scene(irgs, sc)
    p = irgs.TraceParams(k=16, feat_count=F)
    tro, trd = dev(ro), dev(rd)
    tgf, tgd, tgo = dev(gf), dev(gd), dev(go)
    fwd = irgs.trace_forward(S, tro, trd, p, max_hit_ids=96)
    full = irgs.trace_backward(S, tro, trd, p, fwd, tgf, tgd, tgo)
    # (b) linearity over 8 chunks of 8M rays
    parts = None
    step = R // 8
    for lo in range(0, R, step):
        hi = min(R, lo + step)
        sub = {k: v[lo:hi] for k, v in fwd.items()}
        parts = irgs.trace_backward(S, tro[lo:hi], trd[lo:hi], p, sub, tgf[lo:hi], tgd[lo:hi], tgo[lo:hi],
                                    grads=parts)
    torch.cuda.synchronize()
    assert S.status() == 0
    for k in NAMES:
        a, b = full[k].double(), parts[k].double()
        assert float((a - b).norm() / b.norm()) <= 1e-5, k
    del full, parts
    # (a) 512 sampled unambiguous rays: their own backward from the full
    # forward's outputs and hit lists against the oracle's analytic gradient
    rng = np.random.default_rng(31)
    idx = np.sort(rng.choice(R, 1536, replace=False))
    ref_f = oracle.trace(sc, ro[idx], rd[idx], opar(p))
    keep = idx[((ref_f["flags"] & GRAD_FLAGS) == 0) & (ref_f["n_hits"] > 0)][:512]
    assert keep.size == 512
    ti = torch.from_numpy(keep).cuda()
    sub = {k: v[ti].contiguous() for k, v in fwd.items()}
    g = irgs.trace_backward(S, tro[ti], trd[ti], p, sub, tgf[ti], tgd[ti], tgo[ti])
    torch.cuda.synchronize()
    gref = oracle.trace_grad(sc, ro[keep], rd[keep], gf[keep], gd[keep], go[keep], opar(p))
    for k in NAMES:
        a = g[k].cpu().numpy().astype(np.float64).reshape(-1)
        b = gref[k].reshape(-1)
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        el = np.abs(a - b).max() / np.abs(b).max()
        assert rel <= 1e-3 and el <= 1e-3, (k, rel, el)


def test_mc_gradient_full_size_sampled():
    """Per-point albedo and roughness gradients of sampled points (and the
    first and last point) against the oracle; the surfel and environment
    gradients by linearity over two halves of the points."""
    sc = synth.object_scene(n=1_000_000, seed=1002)
    gb = synth.gbuffer_points(640_000, seed=1002)
    env = synth.env_map(seed=1003)
    P = 640_000
    g = np.random.default_rng(1004).normal(size=(P, 3)).astype(np.float32)
    p = irgs.TraceParams(k=16, feat_count=3, t_min=1e-3)
    S = make_scene(irgs, sc)
    tg = [dev(a) for a in gb]
    tenv, tgr = dev(env), dev(g)
    full = irgs.shade_mc_backward(S, *tg, tenv, 32, 32, 2024, p, tgr)
    h = P // 2
    parts = None
    for lo, hi in ((0, h), (h, P)):
        # the halves keep their points' random keys only through a zero
        # upstream gradient on the other half: same call, masked gradient
        gm = tgr.clone()
        gm[:lo] = 0
        gm[hi:] = 0
        parts = irgs.shade_mc_backward(S, *tg, tenv, 32, 32, 2024, p, gm, grads=parts)
    torch.cuda.synchronize()
    assert S.status() == 0
    for k in NAMES + ("env",):
        a, b = full[k].double(), parts[k].double()
        assert float((a - b).norm() / b.norm()) <= 1e-5, k
    # on this scene ~97% of points have some ambiguous ray among their 64, so
    # the per-point gradients are compared on the unambiguous points of a
    # larger sample (flags from the oracle's estimate, then its gradient)
    edges = [0, P - 1]
    idx = np.unique(np.concatenate([np.random.default_rng(6).choice(P, 600, replace=False), edges]))
    f = oracle.shade(sc, *(a[idx] for a in gb), env, 32, 32, 2024, opar(p), margins=oracle.Margins(t_abs=2e-8),
                     point_ids=idx)
    idx = idx[f["flags"] == 0]
    assert idx.size >= 8, idx.size
    sub = [a[idx] for a in gb]
    ref = oracle.shade_grad(sc, *sub, env, 32, 32, 2024, opar(p), g[idx], point_ids=idx, want_env=False)
    for name in ("albedo", "rough"):
        a = full[name].cpu().numpy().astype(np.float64)[idx]
        b = ref[name]
        err = np.abs(a - b).reshape(a.shape[0], -1).max(1) / np.maximum(1.0, np.abs(b).reshape(b.shape[0], -1).max(1))
        assert err.max() <= 1e-3, (name, err.max())


def test_relight_full_size_sampled():
    """Relighting at full size: sampled points and the first and last point
    against the oracle (same point keys), flagged points inside their
    admissible range."""
    sc = synth.object_scene(n=1_000_000, seed=1002)
    gb = synth.gbuffer_points(640_000, seed=1002)
    env = synth.env_map(seed=1005)
    P = 640_000
    p = irgs.TraceParams(k=16, feat_offset=3, feat_count=7, t_min=1e-3)
    S = make_scene(irgs, sc)
    E = irgs.EnvMap(dev(env))
    out = irgs.relight(S, E, *(dev(a) for a in gb), 64, 2025, p)
    torch.cuda.synchronize()
    assert S.status() == 0
    rgb = out["rgb"].cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(rgb)) and np.all(rgb >= 0)
    edges = [0, P - 1]
    idx = np.unique(np.concatenate([np.random.default_rng(8).choice(P, 14, replace=False), edges]))
    sub = [a[idx] for a in gb]
    margins = oracle.Margins(t_abs=2e-8)       # secondary rays start on the surface (as for shading)
    ref = oracle.relight(sc, *sub, env, 64, 2025, opar(p), margins=margins, point_ids=idx)
    g = rgb[idx]
    err = np.abs(g - ref["rgb"]).max(1) / np.maximum(1.0, np.abs(ref["rgb"]).max(1))
    ok = ref["flags"] == 0
    assert np.all(err[ok] <= 1e-4), (err, ref["flags"])
    assert (err <= 1e-4).mean() >= 0.9, err
    # most points have an ambiguous ray among their 64: inside their range
    fl = np.nonzero(~ok)[0]
    if fl.size:
        b = oracle.relight_bounds(sc, *(a[fl] for a in sub), env, 64, 2025, opar(p), margins=margins,
                                  point_ids=idx[fl])
        tol = 1e-4 * np.maximum(1.0, np.abs(ref["rgb"][fl]).max(1))[:, None]
        assert np.all((g[fl] >= b["lo"] - tol) & (g[fl] <= b["hi"] + tol)), (g[fl], b)
    E.close()


def _inside(got, lo, hi, ref_rgb):
    tol = 1e-4 * np.maximum(1.0, np.abs(ref_rgb).max(1))[:, None]
    return np.all((got >= lo - tol) & (got <= hi + tol), axis=1)


def test_wavefront_chunks_above_2_26_rays():
    """1.1M points x 64 samples = 70.4M rays span two wavefront chunks
    (whole points, 2^26 rays = 1,048,576 points per chunk). Shading: 600
    points around the boundary plus the first and last point against the
    oracle (unflagged ones element by element, the flagged ones next to the
    boundary inside their admissible range); the gradient's per-point albedo
    and roughness on the unflagged ones on both sides; relighting on the
    points next to the boundary, the first and the last."""
    sc = synth.object_scene(n=1_000_000, seed=1002)
    P = 1_100_000
    gb = synth.gbuffer_points(P, seed=1006)
    env = synth.env_map(seed=1003)
    pc = (1 << 26) // 64
    near = np.arange(pc - 300, pc + 300)
    idx = np.concatenate([[0], near, [P - 1]])
    p = irgs.TraceParams(k=16, feat_count=3, t_min=1e-3)
    margins = oracle.Margins(t_abs=2e-8)
    S = make_scene(irgs, sc)
    tg = [dev(a) for a in gb]
    rgb = irgs.shade_mc(S, *tg, dev(env), 32, 32, 2024, p)["rgb"].cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert S.status() == 0
    sub = [a[idx] for a in gb]
    ref = oracle.shade(sc, *sub, env, 32, 32, 2024, opar(p), margins=margins, point_ids=idx)
    ok = ref["flags"] == 0
    err = np.abs(rgb[idx] - ref["rgb"]).max(1) / np.maximum(1.0, np.abs(ref["rgb"]).max(1))
    assert np.all(err[ok] <= 1e-4), err[ok].max()
    side = idx >= pc
    assert ok[side].sum() >= 2 and ok[~side].sum() >= 2, (ok[side].sum(), ok[~side].sum())
    edge = np.nonzero((np.abs(idx - pc + 0.5) < 3) & ~ok)[0]   # flagged points next to the boundary
    if edge.size:
        b = oracle.shade_bounds(sc, *(a[edge] for a in sub), env, 32, 32, 2024, opar(p), margins=margins,
                                point_ids=idx[edge])
        assert np.all(_inside(rgb[idx[edge]], b["lo"], b["hi"], ref["rgb"][edge])), idx[edge]
    # gradient (same chunking in the backward): per-point albedo / roughness
    g = np.random.default_rng(1007).normal(size=(P, 3)).astype(np.float32)
    grads = irgs.shade_mc_backward(S, *tg, dev(env), 32, 32, 2024, p, dev(g))
    torch.cuda.synchronize()
    assert S.status() == 0
    keep = idx[ok]
    gref = oracle.shade_grad(sc, *(a[keep] for a in gb), env, 32, 32, 2024, opar(p), g[keep], point_ids=keep,
                             want_env=False)
    for name in ("albedo", "rough"):
        a = grads[name].cpu().numpy().astype(np.float64)[keep]
        b = gref[name]
        e = np.abs(a - b).reshape(a.shape[0], -1).max(1) / np.maximum(1.0, np.abs(b).reshape(b.shape[0], -1).max(1))
        assert e.max() <= 1e-3, (name, e.max())
    del grads
    # relighting (its own chunking, the same 2^26 rays per chunk)
    pr = irgs.TraceParams(k=16, feat_offset=3, feat_count=7, t_min=1e-3)
    env2 = synth.env_map(seed=1005)
    E = irgs.EnvMap(dev(env2))
    out = irgs.relight(S, E, *tg, 64, 2025, pr)["rgb"].cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert S.status() == 0
    ridx = np.array([0, pc - 3, pc - 2, pc - 1, pc, pc + 1, pc + 2, P - 1])
    rsub = [a[ridx] for a in gb]
    rref = oracle.relight(sc, *rsub, env2, 64, 2025, opar(pr), margins=margins, point_ids=ridx)
    rok = rref["flags"] == 0
    rerr = np.abs(out[ridx] - rref["rgb"]).max(1) / np.maximum(1.0, np.abs(rref["rgb"]).max(1))
    assert np.all(rerr[rok] <= 1e-4), (rerr, rref["flags"])
    fl = np.nonzero(~rok)[0]
    if fl.size:
        b = oracle.relight_bounds(sc, *(a[fl] for a in rsub), env2, 64, 2025, opar(pr), margins=margins,
                                  point_ids=ridx[fl])
        assert np.all(_inside(out[ridx[fl]], b["lo"], b["hi"], rref["rgb"][fl])), ridx[fl]
    E.close()
