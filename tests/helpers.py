"""Small scene builders shared by the tests (inputs only, no method code)."""
import numpy as np

from scenegen import frames_to_quats


def cam_identity(W=128, H=128, f=64.0, cx=64.0, cy=64.0):
    """Camera at the world origin looking down +z (camera frame = world frame)."""
    return dict(R=np.eye(3, dtype=np.float32), t=np.zeros(3, dtype=np.float32), fx=np.float32(f),
                fy=np.float32(f), cx=np.float32(cx), cy=np.float32(cy), W=W, H=H)


def fronto_scene(centres, scales, opac, texels, quats=None):
    """Splats parallel to the image plane (identity rotation unless given)."""
    n = len(centres)
    q = np.zeros((n, 4), dtype=np.float32)
    q[:, 0] = 1.0
    if quats is not None:
        q = np.asarray(quats, dtype=np.float32)
    tex = np.asarray(texels, dtype=np.float32)
    return dict(means=np.asarray(centres, dtype=np.float32), quats=q,
                scales=np.asarray(scales, dtype=np.float32),
                opacity=np.asarray(opac, dtype=np.float32), texels=tex, T=tex.shape[1])


def twisted_quat(tu, tv, n):
    return frames_to_quats(np.asarray([tu], float), np.asarray([tv], float), np.asarray([n], float))[0]
