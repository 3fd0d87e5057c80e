"""Exact depth ties: hits at the same exact depth are blended in user-index
order (the (tau, index) key of the exact hit order, Sec. 3.2 / Eq. 8), also
where the surfels' Morton order is the reverse of their user order.

The rays run along -z through coplanar surfels with normal +z at z = 0, from
dyadic origins, so every rounding step of the depth is exact on both sides:
the oracle and the kernels both see tau = 3 for each of them. The oracle
flags such rays as ties (its margin test), so these tests compare them
directly instead of through the flag filter."""
import numpy as np
import pytest

import oracle
from tests.helpers import rays, scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_15867_gb300 as irgs  # noqa: E402
from tests.gpu_util import dev, make_scene  # noqa: E402

NAMES = ("means", "quats", "scales", "opacity", "features")


def tie_scene():
    # users 0, 1, 2 coplanar at z = 0 with x = +0.25, -0.25, 0 (Morton order by
    # x: 1, 2, 0); user 3 parallel below them at z = -0.5
    means = [[0.25, 0.0, 0.0], [-0.25, 0.0, 0.0], [0.0, 0.125, 0.0], [0.0, 0.0, -0.5]]
    quats = [[1.0, 0.0, 0.0, 0.0]] * 4
    scales = [[0.4, 0.3], [0.35, 0.45], [0.5, 0.25], [0.6, 0.6]]
    opac = [0.6, 0.45, 0.7, 0.9]
    feats = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [0.5, 0.5, 0.5]]
    return scene(means, quats, scales, opac, feats)


def tie_rays():
    xs = [-0.0625, 0.0, 0.0625, 0.125, -0.125]
    ys = [0.0, 0.03125, -0.0625]
    o = [[x, y, 3.0] for x in xs for y in ys]
    return rays(o, [[0.0, 0.0, -1.0]] * len(o))


def opar(p):
    return oracle.Params(alpha_min=p.alpha_min, alpha_max=p.alpha_max, T_min=p.T_min, t_min=p.t_min,
                         t_max=p.t_max, feat_offset=p.feat_offset, feat_count=p.feat_count)


def test_morton_order_is_not_user_order():
    sc = tie_scene()
    S = make_scene(irgs, sc)
    perm = S.export()[0]
    coplanar = [u for u in perm if u < 3]
    assert coplanar != sorted(coplanar), perm


@pytest.mark.parametrize("k", [1, 4, 8, 16, 32])
@pytest.mark.parametrize("flags", [0, irgs.FLAG_PER_THREAD])
def test_exact_ties_blend_in_user_order(k, flags):
    sc = tie_scene()
    ro, rd = tie_rays()
    S = make_scene(irgs, sc)
    p = irgs.TraceParams(k=k, feat_count=3, flags=flags)
    out = irgs.trace_forward(S, dev(ro), dev(rd), p, max_hit_ids=8)
    torch.cuda.synchronize()
    assert S.status() == 0
    ref = oracle.trace(sc, ro, rd, opar(p), max_ids=8)
    assert np.all(ref["flags"] & oracle.F_TIE)               # every ray meets the exact tie
    assert np.all(ref["tau"][:, 0] == 3.0) and np.all(ref["tau"][:, 1] == 3.0)
    ids = out["hit_ids"].cpu().numpy()
    np.testing.assert_array_equal(ids, ref["ids"])
    np.testing.assert_array_equal(out["n_hits"].cpu().numpy(), ref["n_hits"])
    for key in ("feat", "depth", "opacity"):
        np.testing.assert_allclose(out[key].cpu().numpy(), ref[key], rtol=0, atol=2e-6)
    # the coplanar hits come first, in ascending user index
    for r in range(ids.shape[0]):
        row = [u for u in ids[r] if u >= 0]
        cop = [u for u in row if u < 3]
        assert cop == sorted(cop) and row[:len(cop)] == cop, row


@pytest.mark.parametrize("saved", [0, 8])
def test_exact_tie_gradients_follow_user_order(saved):
    """The backward's replay (no saved list) and its listed form walk the
    ties in the same (tau, user index) order as the oracle's gradient."""
    sc = tie_scene()
    ro, rd = tie_rays()
    R = ro.shape[0]
    rng = np.random.default_rng(3)
    gf = rng.normal(size=(R, 3)).astype(np.float32)
    gd = rng.normal(size=R).astype(np.float32)
    go = rng.normal(size=R).astype(np.float32)
    S = make_scene(irgs, sc)
    p = irgs.TraceParams(k=8, feat_count=3)
    fwd = irgs.trace_forward(S, dev(ro), dev(rd), p, max_hit_ids=saved)
    g = irgs.trace_backward(S, dev(ro), dev(rd), p, fwd, dev(gf), dev(gd), dev(go))
    torch.cuda.synchronize()
    assert S.status() == 0
    gref = oracle.trace_grad(sc, ro, rd, gf, gd, go, opar(p))
    for k in NAMES:
        a = g[k].cpu().numpy().astype(np.float64).reshape(-1)
        b = gref[k].reshape(-1)
        assert np.abs(a - b).max() <= 1e-4 * max(1.0, np.abs(b).max()), (k, a, b)
