"""The allocation-free LBVH build (irgs_build_lbvh_noalloc) against the
regular build (irgs_build_scene + irgs_scene_export).

That entry point exists for callers that cannot let the library allocate
device memory (an application that owns all GPU memory through its own
arena, or a loop that cannot afford the synchronisation of cudaMalloc). It
works out of one fixed device array inside the library and writes its
results into buffers the caller allocates; here torch allocates them. The
test calls it twice in a row, on two different surfel clouds, so stale
contents of the shared array would show up, and checks both results
against the regular build of the same surfels. It also checks that a cloud
above the stated maximum is refused."""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_15867_gb300 as irgs  # noqa: E402
from paper_2412_15867_gb300 import _build, _lib  # noqa: E402

MAX_SURFELS = 32768   # IRGS_NOALLOC_MAX_SURFELS in include/irgs.h


@pytest.fixture(scope="module")
def L():
    _build.build()
    return _lib.lib()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _noalloc_build(L, sc, alpha_min=1 / 255):
    n = sc.n
    means, quats, scales, opac = (_dev(a) for a in sc.arrays()[:4])
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda:0")
    keys = torch.empty(max(n, 1), dtype=torch.int32, device="cuda:0")
    nodes = torch.empty((max(n - 1, 1), 16), dtype=torch.float32, device="cuda:0")
    boxes = torch.empty((max(n, 1), 6), dtype=torch.float32, device="cuda:0")
    s = _lib.Surfels(means.data_ptr(), quats.data_ptr(), scales.data_ptr(), opac.data_ptr(), None, n, 0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    dev0 = torch.cuda.current_device()
    st = L.irgs_build_lbvh_noalloc(C.byref(s), alpha_min, C.c_void_p(perm.data_ptr()),
                                   C.c_void_p(keys.data_ptr()), C.c_void_p(nodes.data_ptr()),
                                   C.c_void_p(boxes.data_ptr()), stream)
    assert torch.cuda.current_device() == dev0
    if st == 0:
        bits = C.c_uint32(99)
        # the build's device-side status word (0: the hierarchy passed its bounds)
        assert L.irgs_build_lbvh_noalloc_status(0, stream, C.byref(bits)) == 0 and bits.value == 0
        assert torch.cuda.current_device() == dev0
    torch.cuda.synchronize()
    return st, (perm.cpu().numpy()[:n], keys.cpu().numpy().view(np.uint32)[:n], nodes.cpu().numpy(),
                boxes.cpu().numpy()[:n])


def _regular_build(sc):
    S = irgs.Scene(*(_dev(a) for a in sc.arrays()), alpha_min=1 / 255)
    out = S.export()
    S.close()
    return out


def test_noalloc_build_matches_regular_build_twice(L):
    clouds = [synth.object_scene(n=20_000, seed=301), synth.tiny_scene(seed=302, n=MAX_SURFELS)]
    for sc in clouds:
        st, got = _noalloc_build(L, sc)
        assert st == 0, _lib.STATUS.get(st)
        ref = _regular_build(sc)
        for name, a, b in zip(("perm", "keys", "nodes", "leaf_boxes"), got, ref):
            assert a.shape == b.shape, name
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), name


def test_noalloc_build_refuses_clouds_above_its_capacity(L):
    sc = synth.tiny_scene(seed=303, n=MAX_SURFELS + 1)
    st, _ = _noalloc_build(L, sc)
    assert _lib.STATUS.get(st) == "IRGS_ERR_INVALID_ARG"
