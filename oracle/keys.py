"""FP32 specification of splat culling, tile binning and depth keys.

Test infrastructure (see the package header).  The paper relies on the
2DGS/3DGS global sort of splats by tile and depth (supplementary Sec. 3,
"global sorting"); it does not print the binning rule, so this module fixes it
as an exact FP32 operation order that the GPU preprocess reproduces
operation for operation.  Every value below is float32 and every operation is
a single correctly rounded IEEE op (numpy float32 ufuncs: no fused
multiply-add, no transcendental function), so the key list is bit-exact.

Per splat k with mean p, quaternion q = (w,x,y,z), linear scales (s_u, s_v),
opacity o, and a camera (R world->camera row-major, t, fx, fy, cx, cy, W, H):

  1. |q| = sqrt(((w*w + x*x) + y*y) + z*z);  w,x,y,z /= |q|
  2. rotation columns (Sec. 3.1: t_u, t_v and n = t_u x t_v):
       t_u = (1 - 2(yy + zz), 2(xy + wz), 2(xz - wy))
       t_v = (2(xy - wz), 1 - 2(xx + zz), 2(yz + wx))
       n   = (2(xz + wy), 2(yz - wx), 1 - 2(xx + yy))
  3. du = (3 s_u) * t_u, dv = (3 s_v) * t_v   (the 3-sigma support, Sec. 3.3)
  4. corners c = (p +- du) +- dv in the order (-,-), (+,-), (-,+), (+,+)
  5. camera coordinates X_r = ((R_r0 c_0 + R_r1 c_1) + R_r2 c_2) + t_r
  6. cull if any corner has Z <= 0.2 (near plane)
  7. pixel coordinates x = fx * (X/Z) + cx, y = fy * (Y/Z) + cy
  8. tile rect (16x16 tiles): tx0 = max(0, floor(xmin/16)),
     tx1 = min(tiles_x - 1, floor(xmax/16)), same for y; cull if empty
  9. cull if o < (float)(1/255)
 10. depth z = ((R_20 p_0 + R_21 p_1) + R_22 p_2) + t_2; cull if z <= 0.2
 11. one key per covered tile: key = (tile << 32) | float_bits(z),
     tile = ty * tiles_x + tx; keys sorted ascending, equal keys by splat id.

Because the perspective image of the planar support square is the convex
quad of its projected corners, the corner bounding box bounds every pixel
the splat can cover; pixel centres are half-integers and tile edges integers,
so an FP32 error below half a pixel cannot drop a covered pixel's tile.

Parity: pinned by the brute-force test (every contributing pixel/splat pair
of the FP64 renderer lies in the pixel's tile list) and by the FP64 corner
comparison in tests/test_oracle_keys.py.
"""
from __future__ import annotations

import numpy as np

TILE = 16
NEAR = np.float32(0.2)
ALPHA_MIN = np.float32(1.0 / 255.0)

f32 = np.float32


def rotation_columns_f32(quats: np.ndarray):
    """Steps 1-2: normalised quaternion -> (t_u, t_v, n), each [N,3] float32."""
    q = quats.astype(np.float32)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    nrm = np.sqrt(((w * w + x * x) + y * y) + z * z)
    w, x, y, z = w / nrm, x / nrm, y / nrm, z / nrm
    xx, yy, zz = x * x, y * y, z * z
    xy, xz, yz = x * y, x * z, y * z
    wx, wy, wz = w * x, w * y, w * z
    one, two = f32(1.0), f32(2.0)
    tu = np.stack([one - two * (yy + zz), two * (xy + wz), two * (xz - wy)], 1)
    tv = np.stack([two * (xy - wz), one - two * (xx + zz), two * (yz + wx)], 1)
    n = np.stack([two * (xz + wy), two * (yz - wx), one - two * (xx + yy)], 1)
    return tu, tv, n


def _to_cam(R, t, c):
    """Step 5 for points c [...,3] -> camera coordinates (float32)."""
    out = []
    for r in range(3):
        out.append(((R[r, 0] * c[..., 0] + R[r, 1] * c[..., 1]) + R[r, 2] * c[..., 2]) + t[r])
    return np.stack(out, -1)


def splat_view_f32(scene: dict, cam: dict) -> dict:
    """Steps 1-10 for every splat.  Returns float32 corner pixel coordinates,
    the tile rect (inclusive), the depth, its bits and the visibility flag."""
    R = cam["R"].astype(np.float32)
    t = cam["t"].astype(np.float32)
    fx, fy, cx, cy = (f32(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    W, H = int(cam["W"]), int(cam["H"])
    tiles_x, tiles_y = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    p = scene["means"].astype(np.float32)
    s = scene["scales"].astype(np.float32)
    o = scene["opacity"].astype(np.float32)
    tu, tv, _ = rotation_columns_f32(scene["quats"])
    three = f32(3.0)
    du = (three * s[:, 0:1]) * tu
    dv = (three * s[:, 1:2]) * tv
    corners = np.stack([(p - du) - dv, (p + du) - dv, (p - du) + dv, (p + du) + dv], 1)  # [N,4,3]
    Xc = _to_cam(R, t, corners)
    Z = Xc[..., 2]
    front = np.all(Z > NEAR, axis=1)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        px = fx * (Xc[..., 0] / Z) + cx
        py = fy * (Xc[..., 1] / Z) + cy
    xmin, xmax = px.min(1), px.max(1)
    ymin, ymax = py.min(1), py.max(1)
    sixteenth = f32(1.0 / TILE)  # exact power of two: x/16 == x*(1/16)
    with np.errstate(invalid="ignore", over="ignore"):
        tx0 = np.maximum(f32(0.0), np.floor(xmin * sixteenth))
        tx1 = np.minimum(f32(tiles_x - 1), np.floor(xmax * sixteenth))
        ty0 = np.maximum(f32(0.0), np.floor(ymin * sixteenth))
        ty1 = np.minimum(f32(tiles_y - 1), np.floor(ymax * sixteenth))
    nonempty = (tx0 <= tx1) & (ty0 <= ty1)
    depth = _to_cam(R, t, p)[..., 2]
    visible = front & nonempty & (o >= ALPHA_MIN) & (depth > NEAR)
    rect = np.zeros((p.shape[0], 4), dtype=np.int64)
    vis = visible
    rect[vis, 0] = tx0[vis].astype(np.int64)
    rect[vis, 1] = tx1[vis].astype(np.int64)
    rect[vis, 2] = ty0[vis].astype(np.int64)
    rect[vis, 3] = ty1[vis].astype(np.int64)
    return dict(visible=visible, rect=rect, depth=depth.astype(np.float32),
                depth_bits=depth.astype(np.float32).view(np.uint32), corners_px=np.stack([px, py], -1),
                tiles_x=tiles_x, tiles_y=tiles_y)


def build_keys(scene: dict, cam: dict, view=None) -> dict:
    """Step 11: the sorted (key, splat id) list and per-tile [start, end).

    Returns keys (uint64 [K]), ids (uint32 [K]), tile_ranges (int64 [tiles, 2]),
    plus the per-splat data of :func:`splat_view_f32`.
    """
    sv = view if view is not None else splat_view_f32(scene, cam)
    vis_ids = np.nonzero(sv["visible"])[0]
    rect = sv["rect"][vis_ids]
    nx = rect[:, 1] - rect[:, 0] + 1
    ny = rect[:, 3] - rect[:, 2] + 1
    cnt = nx * ny
    K = int(cnt.sum())
    ids = np.repeat(vis_ids, cnt).astype(np.uint32)
    start = np.repeat(np.cumsum(cnt) - cnt, cnt)
    local = np.arange(K, dtype=np.int64) - start
    nx_r = np.repeat(nx, cnt)
    tx = np.repeat(rect[:, 0], cnt) + local % nx_r
    ty = np.repeat(rect[:, 2], cnt) + local // nx_r
    tile = ty * sv["tiles_x"] + tx
    keys = (tile.astype(np.uint64) << np.uint64(32)) | sv["depth_bits"][ids].astype(np.uint64)
    # ascending key, ties by splat id (ids are emitted in ascending order, so a
    # stable sort on the key alone gives that tie order)
    order = np.argsort(keys, kind="stable")
    keys, ids = keys[order], ids[order]
    ntiles = sv["tiles_x"] * sv["tiles_y"]
    tile_sorted = (keys >> np.uint64(32)).astype(np.int64)
    starts = np.searchsorted(tile_sorted, np.arange(ntiles), side="left")
    ends = np.searchsorted(tile_sorted, np.arange(ntiles), side="right")
    return dict(keys=keys, ids=ids, tile_ranges=np.stack([starts, ends], 1), view=sv)
