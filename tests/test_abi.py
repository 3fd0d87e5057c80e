"""The C-ABI library builds, loads and exports every symbol include/irgs.h
declares; calls that fail validation return codes without touching a GPU."""
import ctypes as C
import math

import pytest

from paper_2412_15867_gb300 import _build, _lib


@pytest.fixture(scope="module")
def L():
    _build.build()
    return _lib.lib()


def test_exports_every_declared_symbol(L):
    names = _lib.declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert L.irgs_abi_version() == 3


def test_status_strings(L):
    assert L.irgs_status_string(0) == b"ok"
    assert L.irgs_status_string(1) == b"invalid argument"
    assert L.irgs_status_string(7) == b"device-side error recorded"
    assert L.irgs_status_string(99) == b"unknown status"


def test_null_arguments_rejected_without_gpu(L):
    h = C.c_void_p()
    assert L.irgs_build_scene(None, 1 / 255, None, C.byref(h)) == 1
    s = _lib.Surfels(None, None, None, None, None, -1, 0)
    assert L.irgs_build_scene(C.byref(s), 1 / 255, None, C.byref(h)) == 1
    s = _lib.Surfels(None, None, None, None, None, 4, 0)      # n > 0 with NULL arrays
    assert L.irgs_build_scene(C.byref(s), 1 / 255, None, C.byref(h)) == 1
    s = _lib.Surfels(None, None, None, None, None, 0, 0)
    assert L.irgs_build_scene(C.byref(s), 0.0, None, C.byref(h)) == 1     # alpha_min must be > 0
    assert L.irgs_build_scene_ex(C.byref(s), 1 / 255, 2, None, C.byref(h)) == 1   # unknown build flag
    p = _lib.TraceParamsC(16, 1 / 255, 0.99, 1e-4, 0.0, math.inf, 0, 3, 0)
    assert L.irgs_trace_forward(None, None, None, 0, C.byref(p), None, None, None, None, None, 0, None) == 1
    assert L.irgs_trace_backward(None, None, None, 0, C.byref(p), None, None, None, None, None, 0,
                                 *([None] * 9)) == 1
    assert L.irgs_shade_mc(None, None, None, None, None, None, 0, None, 1, 1, 1, 1, 0, C.byref(p),
                           None, None, None, None) == 1
    assert L.irgs_destroy_scene(None) == 0
    assert L.irgs_scene_info(None, None, None, None, None) == 1


def test_python_binding_fails_loudly_without_cuda_tensors():
    import torch
    import paper_2412_15867_gb300 as irgs
    z = torch.zeros((4, 3))
    with pytest.raises(ValueError):
        irgs.Scene(z, torch.zeros((4, 4)), torch.ones((4, 2)), torch.ones(4))


@pytest.mark.gpu
def test_entry_points_keep_the_callers_current_device(L):
    """Entry points switch to their scene's device and switch back: the
    caller's current device is the same after every call."""
    import torch
    import numpy as np
    import synth
    import paper_2412_15867_gb300 as irgs
    dev0 = torch.cuda.current_device()
    sc = synth.tiny_scene(seed=5, n=256)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    S = irgs.Scene(*(T(a) for a in sc.arrays()))
    assert torch.cuda.current_device() == dev0
    ro, rd = synth.look_at_rays(synth.tiny_camera(5), (0, 0, 0), 8, 8)
    out = irgs.trace_forward(S, T(ro), T(rd), irgs.TraceParams(k=8, feat_count=3))
    assert torch.cuda.current_device() == dev0
    irgs.trace_backward(S, T(ro), T(rd), irgs.TraceParams(k=8, feat_count=3), out, torch.ones_like(out["feat"]))
    assert torch.cuda.current_device() == dev0
    S.update()
    S.refit()
    assert S.status() == 0
    assert torch.cuda.current_device() == dev0
    S.close()
    assert torch.cuda.current_device() == dev0
