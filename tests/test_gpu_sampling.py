"""The secondary-ray sampler on the GPU (Eq. 15's incident directions:
cosine and GGX half-vector sampling, the stratified uniform directions, and
relighting's environment-importance samples of Eq. 18) against the FP64
oracle's, element by element. Both sides draw the same SplitMix64 uniforms
in integer arithmetic; the directions are FP32 on the GPU and FP64 in the
oracle, so they agree to FP32 rounding (bar 2e-5 per component). Whether a
sample is used (above the horizon) is decided in FP32 on the GPU: the two
sides may differ only where the oracle's direction lies within 1e-4 of the
horizon."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_15867_gb300 as irgs  # noqa: E402
from tests.gpu_util import dev  # noqa: E402


def _points(P, seed):
    x, n, a, r, wo = synth.gbuffer_points(P, seed=seed)
    r = r.copy()
    r[: P // 8] = np.float32(0.05)            # the narrowest lobes of the roughness range
    wo = wo.copy()
    wo[P // 8: P // 4] = -wo[P // 8: P // 4]  # w_o below the surface: the normal flips
    return n, r, wo


@pytest.mark.parametrize("mode,nd,ns", [("split", 32, 32), ("split", 5, 27), ("uniform", 40, 0)])
def test_shading_sample_directions_match_oracle(mode, nd, ns):
    P, seed = 700, 2024
    n, r, wo = _points(P, 61)
    d, v = irgs.shade_sample_rays(dev(n), dev(r), dev(wo), nd, ns, seed, mode=mode)
    torch.cuda.synchronize()
    S = nd + ns
    d = d.cpu().numpy().reshape(P, S, 3).astype(np.float64)
    v = v.cpu().numpy().reshape(P, S).astype(bool)
    rd, rv = oracle.sample_dirs(n, wo, r, nd, ns, seed, mode=1 if mode == "uniform" else 0)
    # the side of the horizon decided differently only next to it
    nn = n / np.linalg.norm(n, axis=1, keepdims=True)
    flip = np.sign(np.sum(nn * wo, axis=1))
    height = np.einsum("psk,pk->ps", rd, nn * flip[:, None])
    differ = v != rv
    assert np.all(np.abs(height[differ]) < 1e-4), height[differ]
    assert differ.mean() < 1e-3
    both = v & rv
    assert both.mean() > 0.8
    err = np.abs(d - rd).max(axis=2)
    assert err[both].max() <= 2e-5, err[both].max()
    np.testing.assert_allclose(np.linalg.norm(d[both], axis=1), 1.0, atol=1e-6)


def test_environment_sample_directions_match_oracle():
    env = synth.env_map(seed=63, height=64, width=128)
    E = irgs.EnvMap(dev(env))
    P, S, seed = 300, 64, 77
    d, pdf, v = irgs.relight_sample_rays(E, P, S, seed)
    torch.cuda.synchronize()
    rd, rp = oracle.env_samples(env, P, S, seed)
    d = d.cpu().numpy().reshape(P, S, 3).astype(np.float64)
    pdf = pdf.cpu().numpy().reshape(P, S).astype(np.float64)
    v = v.cpu().numpy().reshape(P, S).astype(bool)
    assert v.all() and np.all(rp > 0)
    assert np.abs(d - rd).max() <= 2e-5
    np.testing.assert_allclose(pdf, rp, rtol=2e-5)
    E.close()
