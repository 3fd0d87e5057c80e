"""Small scene builders for the tests (no tracer arithmetic here)."""
import numpy as np
from scipy.spatial.transform import Rotation

from synth import Surfels


def quat_wxyz(rot: Rotation) -> np.ndarray:
    xyzw = rot.as_quat()
    return np.array([xyzw[3], xyzw[0], xyzw[1], xyzw[2]])


def frame_of(q_wxyz):
    """(t_u, t_v, n) from SciPy's rotation matrix of q (w,x,y,z)."""
    q = np.asarray(q_wxyz, np.float64)
    m = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    return m[:, 0], m[:, 1], m[:, 2]


def scene(means, quats, scales, opacity, feats) -> Surfels:
    f = lambda a, shp: np.ascontiguousarray(np.asarray(a, np.float64).reshape(shp), np.float32)
    means = f(means, (-1, 3))
    n = means.shape[0]
    feats = np.asarray(feats, np.float64)
    nf = feats.shape[-1] if feats.ndim >= 1 and feats.size == 0 else (feats.size // max(n, 1))
    return Surfels(means, f(quats, (n, 4)), f(scales, (n, 2)), f(opacity, (n,)),
                   f(feats, (n, nf)))


def rays(o, d):
    return (np.ascontiguousarray(np.asarray(o, np.float64).reshape(-1, 3), np.float32),
            np.ascontiguousarray(np.asarray(d, np.float64).reshape(-1, 3), np.float32))
