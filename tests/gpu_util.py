"""Helpers for the GPU parity tests: device upload and the comparison bars.

Bars (forward, composited channels feat/depth/opacity, max abs error per ray):
  * >= 99.9% of all rays within 1e-4;
  * every ray without an ambiguity flag within 2e-3 and with the oracle's
    exact hit count (and hit id sequence where requested);
  * flagged rays (an exact answer within a margin of a discontinuity: the
    alpha cutoff, the 3-sigma support edge, the T_min stop, near-equal depths,
    the ray interval ends, the grazing threshold) must equal, within 1e-4 and
    with the same hit count, one of the outcomes the oracle lists as
    admissible for them (each ambiguous candidate in or out, near-tied hits
    in any order, the stop on either side of T_min); rays with too many
    outcomes to list are counted, bounded, and checked for validity only;
  * every ray is valid: finite, opacity in [0,1], features within
    [0, opacity * max f].
"""
import numpy as np
import torch

import oracle


def dev(a, device="cuda:0"):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def make_scene(irgs, sc, alpha_min=1 / 255):
    return irgs.Scene(*(dev(a) for a in sc.arrays()), alpha_min=alpha_min)


def oracle_reference(sc, ro, rd, params, max_ids=0, max_alts=256):
    """oracle.trace plus, for its flagged rays, the admissible outcomes
    (oracle.trace_alternatives) that assert_forward_parity checks them with."""
    ref = oracle.trace(sc, ro, rd, params, max_ids=max_ids)
    idx = np.nonzero((ref["flags"] & oracle.FORWARD_FLAGS) != 0)[0]
    ref["alt_rays"] = idx
    ref["alts"] = oracle.trace_alternatives(sc, np.asarray(ro)[idx], np.asarray(rd)[idx], params,
                                            max_alts=max_alts)
    return ref


def alternative_errors(out, ref):
    """Per flagged ray: the smallest max-abs error against an admissible
    outcome with the same hit count (inf if none), and the outcome count."""
    idx = ref["alt_rays"]
    A = ref["alts"]
    f = out["feat"].detach().cpu().numpy().astype(np.float64)[idx]
    d = out["depth"].detach().cpu().numpy().astype(np.float64)[idx]
    o = out["opacity"].detach().cpu().numpy().astype(np.float64)[idx]
    e = np.maximum(np.abs(d[:, None] - A["depth"]), np.abs(o[:, None] - A["opacity"]))
    if f.shape[1]:
        e = np.maximum(e, np.abs(f[:, None, :] - A["feat"]).max(axis=2))
    cnt = A["count"]
    slot = np.arange(e.shape[1])[None, :]
    valid = slot < np.where(cnt < 0, 1, cnt)[:, None]
    if "n_hits" in out:          # (the serving path reports no hit counts)
        valid &= A["n_hits"] == out["n_hits"].cpu().numpy()[idx][:, None]
    e = np.where(valid, e, np.inf)
    return e.min(axis=1) if e.size else np.zeros(len(idx)), cnt


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
                          tol_all=2e-3, frac=0.999, max_flagged=None, max_unresolved=1e-3):
    err = forward_errors(out, ref)
    strict = (ref["flags"] & oracle.FORWARD_FLAGS) == 0
    within = err <= tol_frac
    stats = {"rays": int(err.size), "strict": float(strict.mean()), "within_1e-4": float(within.mean()),
             "max_err_strict": float(err[strict].max()) if strict.any() else 0.0,
             "max_err_all": float(err.max()) if err.size else 0.0}
    assert within.mean() >= frac, stats
    assert np.all(err[strict] <= tol_all), stats
    # flagged rays: one of the admissible outcomes, same hit count, within tol_frac
    flagged = np.nonzero(~strict)[0]
    if flagged.size:
        assert "alts" in ref, "flagged rays need the admissible outcomes (gpu_util.oracle_reference)"
        assert np.array_equal(ref["alt_rays"], flagged)
        ealt, cnt = alternative_errors(out, ref)
        resolved = cnt >= 0
        stats.update({"flagged": int(flagged.size), "unresolved": int((~resolved).sum()),
                      "max_err_flagged": float(ealt[resolved].max()) if resolved.any() else 0.0,
                      "max_outcomes": int(cnt.max())})
        bad = flagged[resolved & ~(ealt <= tol_frac)]
        assert bad.size == 0, ("flagged rays match no admissible outcome", bad[:10], ealt[resolved][:10], stats)
        assert (~resolved).sum() <= max_unresolved * err.size, stats
    stats["flagged_frac"] = float(flagged.size / max(err.size, 1))
    if max_flagged is not None:
        assert stats["flagged_frac"] <= max_flagged, stats
    if "n_hits" in out:
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
