"""The binary hierarchy of the scene build (the BVH over the surfel proxies
of Sec. 3.2), made by locally-ordered clustering over the Morton-sorted
leaves, with the Karras radix tree as the fallback for trees too high.

Checked on the exported hierarchy: every leaf and node reached once, every
node box exactly the union of its children's boxes, the same tree from two
builds, a lower total node surface area than the radix tree over the same
sorted keys, balanced pairing of identical surfels, the fallback on a
contrived chain (whose traces must still match the oracle), and the
radix-tree build option: the Karras split of every node's range, and
traces identical to those on the clustered tree."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_15867_gb300 as irgs  # noqa: E402
from tests.gpu_util import dev, make_scene  # noqa: E402


def walk(nodes, boxes):
    """(height, total node surface area, node boxes tight) of the binary tree
    rooted at node 0; asserts that every leaf and node is reached once."""
    n = boxes.shape[0]
    ch = nodes[:, 12:14].view(np.int32)
    seen_leaf = np.zeros(n, np.int32)
    seen_node = np.zeros(max(n - 1, 1), np.int32)
    lo = np.zeros((max(n - 1, 1), 3), np.float32)
    hi = np.zeros((max(n - 1, 1), 3), np.float32)
    order, stack, depth = [], [(0, 1)], 0
    seen_node[0] = 1
    while stack:
        i, d = stack.pop()
        depth = max(depth, d)
        order.append(i)
        for c in ch[i]:
            if c < 0:
                seen_leaf[~c] += 1
            else:
                seen_node[c] += 1
                stack.append((c, d + 1))
    assert np.all(seen_leaf == 1) and np.all(seen_node == 1)
    tight = True
    for i in reversed(order):          # children before parents
        b = []
        for s, c in enumerate(ch[i]):
            stored = nodes[i, 6 * s:6 * s + 6]
            ref = boxes[~c] if c < 0 else np.r_[lo[c], hi[c]]
            tight &= bool(np.array_equal(stored, ref))
            b.append(ref)
        lo[i] = np.minimum(b[0][:3], b[1][:3])
        hi[i] = np.maximum(b[0][3:], b[1][3:])
    e = (hi - lo).astype(np.float64)
    area = float((e[:, 0] * e[:, 1] + e[:, 1] * e[:, 2] + e[:, 2] * e[:, 0]).sum())
    return depth, area, tight


def radix_tree_area(keys, boxes):
    """Total node surface area of the Karras radix tree over the sorted keys
    (ties split by index bits), computed by recursive range splitting."""
    k = keys.astype(np.int64) * (1 << 32) + np.arange(keys.size)
    total, stack = 0.0, [(0, keys.size - 1)]
    while stack:
        f, l = stack.pop()
        if f == l:
            continue
        e = (boxes[f:l + 1, 3:].max(0) - boxes[f:l + 1, :3].min(0)).astype(np.float64)
        total += e[0] * e[1] + e[1] * e[2] + e[2] * e[0]
        b = int(k[f] ^ k[l]).bit_length() - 1
        sp = f + int(np.argmax((k[f:l + 1] >> b) & 1)) - 1
        stack += [(f, sp), (sp + 1, l)]
    return total


def test_clustered_hierarchy_is_valid_tight_deterministic_and_better_than_radix_tree():
    sc = synth.object_scene(n=40_000, seed=501)
    S1, S2 = make_scene(irgs, sc), make_scene(irgs, sc)
    torch.cuda.synchronize()
    assert S1.status() == 0
    perm, keys, nodes, boxes = S1.export()
    for a, b in zip((perm, keys, nodes, boxes), S2.export()):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    height, area, tight = walk(nodes, boxes)
    assert tight
    assert height <= 60
    radix = radix_tree_area(keys, boxes)
    assert area < 0.9 * radix, (area, radix)
    print({"height": height, "area / radix-tree area": area / radix})


def test_identical_surfels_pair_up_into_a_balanced_tree():
    n = 5000
    sc = scene(np.tile([[0.1, -0.2, 0.3]], (n, 1)), np.tile([[1.0, 0, 0, 0]], (n, 1)), np.tile([[0.2, 0.1]], (n, 1)),
               np.full(n, 0.6), np.tile([[0.5, 0.5, 0.5]], (n, 1)))
    S = make_scene(irgs, sc)
    _, _, nodes, boxes = S.export()
    height, _, tight = walk(nodes, boxes)
    assert tight and height == math.ceil(math.log2(n))


def test_a_chain_too_high_falls_back_to_the_radix_tree():
    """Surfels on a diagonal with geometrically growing size: each round can
    only merge the two smallest clusters, so clustering would give a chain of
    height n - 1; the build keeps the radix tree instead (equal Morton codes:
    split by index, height ceil(log2 n))."""
    n = 200
    s = 1.25 ** np.arange(n)
    sc = scene(np.c_[s, s, s], np.tile([[1.0, 0, 0, 0]], (n, 1)), np.c_[0.1 * s, 0.1 * s], np.full(n, 0.5),
               np.random.default_rng(3).uniform(0, 1, size=(n, 3)))
    S = make_scene(irgs, sc)
    perm, keys, nodes, boxes = S.export()
    torch.cuda.synchronize()
    assert S.status() == 0
    height, area, tight = walk(nodes, boxes)
    assert tight and height <= 62
    ro = np.tile(np.array([[0.0, 0.0, 0.0]], np.float32), (256, 1))
    rd = np.random.default_rng(4).normal(size=(256, 3)).astype(np.float32)
    rd[:, :] = np.abs(rd) + 0.2
    rd /= np.linalg.norm(rd, axis=1, keepdims=True)
    p = irgs.TraceParams(k=8, feat_count=3)
    out = irgs.trace_forward(S, dev(ro), dev(rd), p)
    ref = oracle.trace(sc, ro, rd, oracle.Params(alpha_min=p.alpha_min, alpha_max=p.alpha_max, T_min=p.T_min,
                                                 t_min=p.t_min, t_max=p.t_max, feat_offset=0, feat_count=3))
    # depths reach ~1e19 here: depth relative, the blended values absolute
    ok = ref["flags"] == 0
    assert ok.mean() > 0.9
    d = out["depth"].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(d - ref["depth"])[ok] <= 1e-5 * np.maximum(1.0, np.abs(ref["depth"][ok])))
    for k in ("opacity", "feat"):
        a = out[k].cpu().numpy().astype(np.float64).reshape(256, -1)
        assert np.all(np.abs(a - ref[k].reshape(256, -1))[ok] <= 1e-4), k
    assert np.array_equal(out["n_hits"].cpu().numpy()[ok], ref["n_hits"][ok])
    assert int(out["n_hits"].sum()) > 0


def leaf_ranges(nodes, n):
    """(first, last) leaf index under every internal node of the exported tree."""
    ch = nodes[:, 12:14].view(np.int32)
    first = np.zeros(max(n - 1, 1), np.int64)
    last = np.zeros(max(n - 1, 1), np.int64)
    order, stack = [], [0]
    while stack:
        i = stack.pop()
        order.append(i)
        stack += [c for c in ch[i] if c >= 0]
    for i in reversed(order):
        r = [(~c, ~c) if c < 0 else (first[c], last[c]) for c in ch[i]]
        first[i], last[i] = r[0][0], r[1][1]
        assert r[0][1] + 1 == r[1][0]          # children cover adjacent ranges, left first
    return ch, first, last


def test_radix_tree_option_builds_the_karras_tree_and_traces_identically():
    sc = synth.object_scene(n=20_000, seed=511)
    sc = sc.subset(np.concatenate([np.arange(sc.n), np.arange(300)]))     # equal Morton codes occur
    arrays = [dev(a) for a in sc.arrays()]
    R = irgs.Scene(*arrays, hierarchy="radix")
    Cl = irgs.Scene(*arrays)
    pr, kr, nr, br = R.export()
    pc, kc, nc, bc = Cl.export()
    assert np.array_equal(pr, pc) and np.array_equal(kr, kc) and np.array_equal(br, bc)
    n = sc.n
    height, _, tight = walk(nr, br)
    assert tight and height <= 62
    # every node splits its range where the radix tree does: at the highest
    # bit in which the extended keys (Morton code, then index) of its ends differ
    ch, first, last = leaf_ranges(nr, n)
    k = kr.astype(np.int64) * (1 << 32) + np.arange(n)
    for i in range(n - 1):
        f, l = first[i], last[i]
        b = int(k[f] ^ k[l]).bit_length() - 1
        split = f + int(np.count_nonzero(((k[f:l + 1] >> b) & 1) == 0)) - 1
        c0 = ch[i, 0]
        assert (~c0 if c0 < 0 else last[c0]) == split, i
    ro, rd = synth.camera_batch_rays(synth.hemisphere_cameras(2, seed=512), 64, 48, tile=(8, 4))
    for flags in (0, irgs.FLAG_PER_THREAD):
        p = irgs.TraceParams(k=16, feat_count=10, flags=flags)
        a = irgs.trace_forward(R, dev(ro), dev(rd), p, max_hit_ids=64)
        b = irgs.trace_forward(Cl, dev(ro), dev(rd), p, max_hit_ids=64)
        for key in ("feat", "depth", "opacity", "n_hits", "hit_ids"):
            assert torch.equal(a[key], b[key]), (flags, key)
    # the choice survives an in-place rebuild
    R.update(means=arrays[0] + 0.01)
    _, _, nr2, br2 = R.export()
    _, first2, last2 = leaf_ranges(nr2, n)
    assert walk(nr2, br2)[2]
    with pytest.raises(ValueError):
        irgs.Scene(*arrays, hierarchy="octree")
