"""GPU relighting query vs the oracle (supplementary "Relighting details",
Eq. 18): the pre-integrated maps element by element, then the per-point
estimate. Maps: FP32 block sums of the same texel terms (relative 2e-5 of
the map's largest value), the BRDF table within 2e-5, the FP64 sampling
cdfs to 1e-12 relative. Estimates: as for the shading estimate, relative
above 1: |rgb - ref| <= 1e-4 max(1, |ref|) on >= 99% of points and 2e-3 on
every point whose traced rays carry no ambiguity flag."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_15867_gb300 as irgs  # noqa: E402
from tests.gpu_util import dev, make_scene  # noqa: E402

MAT = dict(feat_offset=3, feat_count=7)   # albedo, roughness, normal of the object scene


def opar(p):
    return oracle.Params(alpha_min=p.alpha_min, alpha_max=p.alpha_max, T_min=p.T_min, t_min=p.t_min,
                         t_max=p.t_max, feat_offset=p.feat_offset, feat_count=p.feat_count)


@pytest.mark.parametrize("h,w", [(64, 128), (37, 50)])
def test_maps_match_oracle(h, w):
    env = synth.env_map(seed=401, height=h, width=w)
    E = irgs.EnvMap(dev(env))
    g = E.export()
    ref = oracle.relight_maps(env)
    for k in ("irr", "pref"):
        scale = np.abs(ref[k]).max()
        assert np.abs(g[k] - ref[k]).max() <= 2e-5 * scale, k
    assert np.abs(g["lut"] - ref["lut"]).max() <= 2e-5
    np.testing.assert_allclose(g["row_cdf"], ref["row_cdf"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(g["col_cdf"], ref["col_cdf"], rtol=1e-12, atol=1e-300)
    E.close()


def check(out, ref, frac=0.99, bounds=None):
    """Unflagged points at the shading bars; flagged points (if `bounds`, the
    oracle's relight_bounds of the flagged points) inside their admissible
    range within 1e-4 max(1, |ref|)."""
    g = out["rgb"].cpu().numpy().astype(np.float64)
    err = np.abs(g - ref["rgb"]).max(1) / np.maximum(1.0, np.abs(ref["rgb"]).max(1))
    ok = ref["flags"] == 0
    st = {"points": int(err.size), "unflagged": float(ok.mean()), "max_err": float(err.max()),
          "max_err_unflagged": float(err[ok].max()) if ok.any() else None, "within": float((err <= 1e-4).mean())}
    assert (err <= 1e-4).mean() >= frac, st
    assert np.all(err[ok] <= 2e-3), st
    if bounds is not None:
        fl = np.nonzero(~ok)[0]
        tol = 1e-4 * np.maximum(1.0, np.abs(ref["rgb"][fl]).max(1))[:, None]
        inside = (g[fl] >= bounds["lo"] - tol) & (g[fl] <= bounds["hi"] + tol)
        st["flagged"] = int(fl.size)
        assert np.all(inside), ("flagged points outside their admissible range", fl[~inside.all(1)], st)
    v = out["vis"].cpu().numpy()
    assert np.all(np.abs(v - ref["vis"])[ok] <= 1e-4), st
    ind = out["ind"].cpu().numpy()
    assert np.all(np.abs(ind - ref["ind"]).max(1)[ok] <= 1e-4 * np.maximum(1, np.abs(ref["ind"]).max(1)[ok])), st
    return st


@pytest.mark.parametrize("k,S,flags", [(16, 64, 0), (8, 13, 0), (16, 64, 1)])
def test_relight_matches_oracle_object_scene(k, S, flags):
    sc = synth.object_scene(n=20_000, seed=411)
    x, n, a, r, wo = synth.gbuffer_points(48, seed=412)
    env = synth.env_map(seed=413, height=64, width=128)
    p = irgs.TraceParams(k=k, t_min=1e-3, flags=flags, **MAT)
    S_ = make_scene(irgs, sc)
    E = irgs.EnvMap(dev(env))
    out = irgs.relight(S_, E, dev(x), dev(n), dev(a), dev(r), dev(wo), S, 77, p, want_aux=True)
    torch.cuda.synchronize()
    assert S_.status() == 0
    ref = oracle.relight(sc, x, n, a, r, wo, env, S, 77, opar(p))
    fl = np.nonzero(ref["flags"] != 0)[0]
    b = (oracle.relight_bounds(sc, x[fl], n[fl], a[fl], r[fl], wo[fl], env, S, 77, opar(p), point_ids=fl)
         if fl.size else None)
    print(check(out, ref, bounds=b))


def test_relight_furnace_and_visibility_in_an_empty_scene():
    z = np.zeros((0, 3), np.float32)
    empty = scene(z, np.zeros((0, 4)), np.zeros((0, 2)), np.zeros(0), np.zeros((0, 10)))
    L = np.array([1.5, 1.0, 0.5], np.float32)
    env = np.tile(L, (16, 32, 1)).astype(np.float32)
    x, n, a, r, wo = synth.gbuffer_points(32, seed=421)
    p = irgs.TraceParams(k=8, t_min=1e-3, **MAT)
    S_ = make_scene(irgs, empty)
    E = irgs.EnvMap(dev(env))
    out = irgs.relight(S_, E, dev(x), dev(n), dev(a), dev(r), dev(wo), 40, 5, p, want_aux=True)
    ref = oracle.relight(empty, x, n, a, r, wo, env, 40, 5, opar(p))
    check(out, ref, frac=1.0)
    np.testing.assert_allclose(out["vis"].cpu().numpy(), 1.0)
    assert float(out["ind"].abs().max()) == 0.0


def test_relight_argument_checks():
    sc = synth.object_scene(n=1_000, seed=431)
    S_ = make_scene(irgs, sc)
    E = irgs.EnvMap(dev(synth.env_map(seed=432, height=8, width=16)))
    x, n, a, r, wo = synth.gbuffer_points(4, seed=433)
    args = (dev(x), dev(n), dev(a), dev(r), dev(wo))
    with pytest.raises(irgs.IrgsError):
        irgs.relight(S_, E, *args, 8, 0, irgs.TraceParams(k=8, t_min=1e-3, feat_offset=0, feat_count=3))
    with pytest.raises(irgs.IrgsError):
        irgs.relight(S_, E, *args, 0, 0, irgs.TraceParams(k=8, t_min=1e-3, **MAT))
    with pytest.raises(irgs.IrgsError):
        irgs.relight(S_, E, *args, 8, 0, irgs.TraceParams(k=8, t_min=0.0, **MAT))


def test_relight_wavefront_and_fused_agree():
    sc = synth.object_scene(n=10_000, seed=441)
    x, n, a, r, wo = synth.gbuffer_points(70, seed=442)
    env = synth.env_map(seed=443, height=32, width=64)
    S_ = make_scene(irgs, sc)
    E = irgs.EnvMap(dev(env))
    args = (dev(x), dev(n), dev(a), dev(r), dev(wo), 45, 3)
    o1 = irgs.relight(S_, E, *args, irgs.TraceParams(k=16, t_min=1e-3, **MAT), want_aux=True)
    o2 = irgs.relight(S_, E, *args, irgs.TraceParams(k=16, t_min=1e-3, flags=irgs.FLAG_PER_THREAD, **MAT),
                      want_aux=True)
    torch.cuda.synchronize()
    assert S_.status() == 0
    for k in o1:
        assert torch.allclose(o1[k], o2[k], rtol=1e-6, atol=1e-6), k
