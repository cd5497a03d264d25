"""Small scene builders and oracle-comparison helpers shared by the tests (no method code)."""
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


def admissible_errors(gpu, ref, key="rgba"):
    """Per-pixel max-abs error of a GPU output against the oracle's admissible
    results: the definition's value, or, where exactly one discrete decision
    of the pixel (support edge, alpha threshold, termination, orientation)
    lies within FP32 error of flipping, the value with that decision flipped
    (ref["alt"]).  Works for [..., C] and [...] arrays (rgba, X, A, T, Z)."""
    g = np.asarray(gpu, dtype=np.float64)
    r = ref[key].detach().numpy() if hasattr(ref[key], "detach") else np.asarray(ref[key])
    a = ref["alt"][key]
    a = a.detach().numpy() if hasattr(a, "detach") else np.asarray(a)
    e0, e1 = np.abs(g - r), np.abs(g - a)
    if e0.ndim > np.asarray(ref["ambiguous"]).ndim:
        e0, e1 = e0.max(-1), e1.max(-1)
    return np.minimum(e0, e1)


def check_admissible(gpu, ref, tol=1e-4, max_masked=1e-3, label="", key="rgba"):
    """GPU output within `tol` of an admissible oracle result on every pixel
    that has one; pixels with several decisions near their switching points
    (no unique pair of results) are masked, and their fraction is printed
    and bounded by `max_masked`.  Returns the statistics."""
    amb = ref["ambiguous"].numpy() if hasattr(ref["ambiguous"], "numpy") else np.asarray(ref["ambiguous"])
    alt = ref["alt_mask"] if "alt_mask" in ref else ref["alt"]["mask"]
    alt = alt.numpy() if hasattr(alt, "numpy") else np.asarray(alt)
    err = admissible_errors(gpu, ref, key)
    frac = float(amb.mean()) if amb.size else 0.0
    ok = ~amb
    stats = dict(pixels=int(amb.size), masked=int(amb.sum()), masked_frac=frac, two_results=int(alt.sum()),
                 max_err=float(err[ok].max()) if ok.any() else 0.0)
    print(f"[parity] {label} {key}: {stats}")
    assert frac <= max_masked, (label, stats)
    bad = (err > tol) & ok
    assert not bad.any(), (label, int(bad.sum()), float(err[ok].max()), np.argwhere(bad)[:5])
    return stats
