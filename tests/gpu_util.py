"""Helpers for the GPU parity tests: device upload and the comparison bars.

Bars (forward, composited channels feat/depth/opacity, max abs error per ray):
  * >= 99.9% of all rays within 1e-4;
  * every ray without an ambiguity flag within 2e-3 and with the oracle's
    exact hit count (and hit id sequence where requested);
  * flagged rays (an exact answer within a margin of a discontinuity: the
    alpha cutoff, the 3-sigma support edge, the T_min stop, near-equal depths,
    the ray interval ends, the grazing threshold) are checked for validity:
    finite, opacity in [0,1], features within [0, opacity * max f].
"""
import numpy as np
import torch

import oracle


def dev(a, device="cuda:0"):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def make_scene(irgs, sc, alpha_min=1 / 255):
    return irgs.Scene(*(dev(a) for a in sc.arrays()), alpha_min=alpha_min)


def forward_errors(out, ref):
    f = out["feat"].detach().cpu().numpy().astype(np.float64)
    d = out["depth"].detach().cpu().numpy().astype(np.float64)
    o = out["opacity"].detach().cpu().numpy().astype(np.float64)
    e = np.abs(d - ref["depth"])
    e = np.maximum(e, np.abs(o - ref["opacity"]))
    if f.shape[1]:
        e = np.maximum(e, np.abs(f - ref["feat"]).max(axis=1))
    return e


def assert_forward_parity(out, ref, sc_feats=None, feat_offset=0, check_ids=False, tol_frac=1e-4,
                          tol_all=2e-3, frac=0.999):
    err = forward_errors(out, ref)
    strict = (ref["flags"] & oracle.FORWARD_FLAGS) == 0
    within = err <= tol_frac
    stats = {"rays": int(err.size), "strict": float(strict.mean()), "within_1e-4": float(within.mean()),
             "max_err_strict": float(err[strict].max()) if strict.any() else 0.0,
             "max_err_all": float(err.max()) if err.size else 0.0}
    assert within.mean() >= frac, stats
    assert np.all(err[strict] <= tol_all), stats
    nh = out["n_hits"].cpu().numpy()
    bad = np.nonzero(strict & (nh != ref["n_hits"]))[0]
    assert bad.size == 0, ("n_hits differ", bad[:10], nh[bad[:10]], ref["n_hits"][bad[:10]])
    if check_ids:
        gid = out["hit_ids"].cpu().numpy()
        m = gid.shape[1]
        rid = ref["ids"][:, :m]
        badi = np.nonzero(strict & np.any(gid != rid, axis=1))[0]
        assert badi.size == 0, ("hit ids differ", badi[:5], gid[badi[:2]], rid[badi[:2]])
    # validity everywhere
    o = out["opacity"].cpu().numpy()
    f = out["feat"].cpu().numpy()
    assert np.all(np.isfinite(o)) and np.all(np.isfinite(f)) and np.all(np.isfinite(out["depth"].cpu().numpy()))
    assert np.all(o >= -1e-6) and np.all(o <= 1 + 1e-6)
    if sc_feats is not None and f.shape[1]:
        fc = f.shape[1]
        fmax = sc_feats[:, feat_offset:feat_offset + fc].max(axis=0)
        fmin = sc_feats[:, feat_offset:feat_offset + fc].min(axis=0)
        if np.all(fmin >= 0):
            assert np.all(f <= o[:, None] * fmax + 1e-5) and np.all(f >= -1e-5)
    return stats
