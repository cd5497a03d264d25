"""ctypes declarations of libtexsplat.so (include/texsplat.h).

Loading fails loudly when the library has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtexsplat.so")

TS_F32, TS_BF16, TS_F16 = 0, 1, 2
SAMPLERS = {"software": 0, "hw_atlas": 1, "flat": 2}
PACKINGS = {"splat_id": 0, "morton": 1}
NORMAL_ENCODINGS = {"xyz": 0, "xy": 1}
STATUS = {0: "TS_OK", 1: "TS_ERR_ARG", 2: "TS_ERR_OOM", 3: "TS_ERR_CAPACITY", 4: "TS_ERR_CUDA",
          5: "TS_ERR_TIMEOUT", 6: "TS_ERR_STATE"}

EXPORTED = [
    "ts_create_scene", "ts_destroy_scene", "ts_upload_gaussians", "ts_upload_atlas", "ts_upload_envmap",
    "ts_render", "ts_render_views", "ts_render_backward", "ts_release_saved", "ts_saved_sizes",
    "ts_saved_copy_lists", "ts_saved_copy_pixels", "ts_saved_frag_stats", "ts_l1_loss",
    "ts_launch_count", "ts_profile_enable", "ts_profile_report", "ts_last_error", "ts_version",
    "ts_render_noalloc", "ts_scene_info", "ts_server_create", "ts_server_destroy", "ts_server_submit",
    "ts_server_wait", "ts_server_stats", "ts_server_reset_stats", "ts_scene_texels", "ts_scene_set_geometry",
    "ts_adam_update", "ts_measure_fp32_peak", "ts_scene_build_atlas2d", "ts_scene_set_sampler",
    "ts_image_loss", "ts_saved_copy_depth", "ts_normal_loss", "ts_upload_indirect",
    "ts_scene_set_normal_encoding", "ts_scene_envmap", "ts_activate", "ts_activate_backward",
    "ts_selftest_sort_wait", "ts_debug_fail_alloc", "ts_server_batch_log",
    "ts_server_request_bytes",
]


class TsCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("visibility", C.c_void_p)]


class TsGrads(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("means", "quats", "scales", "opacity", "texels", "spec", "irr", "sh")]


class TsFragStats(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("n_evaluated", C.c_int64), ("n_blended", C.c_int64),
                ("n_visible", C.c_int64), ("n_texels_read", C.c_int64), ("n_items_blended", C.c_int64)]


class TsServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64),
                ("failed", C.c_int64), ("batches", C.c_int64), ("mean_batch", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("fps", C.c_double),
                ("mpix_per_s", C.c_double), ("true_ups", C.c_int64), ("over_budget", C.c_int64),
                ("peak_reserved_bytes", C.c_double)]


class TsAdam(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int64)]


class TexSplatError(RuntimeError):
    pass


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise TexSplatError(f"{LIB_PATH} is missing: build it with `python -m paper_2506_13348_b300.build` "
                            "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
    sig = {
        "ts_create_scene": [C.POINTER(vp), i32],
        "ts_destroy_scene": [vp],
        "ts_upload_gaussians": [vp, i64, vp, vp, vp, vp, i32, vp],
        "ts_upload_atlas": [vp, i32, i32, i32, vp, i32, vp],
        "ts_upload_envmap": [vp, i32, i32, vp, i32, vp, i32, vp, i32, i32, vp],
        "ts_render": [vp, C.POINTER(TsCamera), vp, C.POINTER(vp), vp],
        "ts_render_views": [C.POINTER(vp), C.POINTER(TsCamera), i32, C.POINTER(vp), C.POINTER(vp), vp],
        "ts_render_backward": [vp, C.POINTER(vp), C.POINTER(TsGrads), vp],
        "ts_release_saved": [vp],
        "ts_saved_sizes": [vp, C.POINTER(i64), C.POINTER(i64)],
        "ts_saved_copy_lists": [vp, vp, vp, vp, vp],
        "ts_saved_copy_pixels": [vp, i32, vp, vp, vp, vp],
        "ts_saved_frag_stats": [vp, C.POINTER(TsFragStats), vp],
        "ts_l1_loss": [vp, vp, i64, vp, vp, vp],
        "ts_profile_enable": [i32],
        "ts_profile_report": [C.c_char_p, C.c_size_t],
        "ts_render_noalloc": [i64, vp, vp, vp, vp, i32, vp, i32, i32, vp, i32, vp, i32, vp,
                              C.POINTER(TsCamera), vp, vp],
        "ts_scene_info": [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32)],
        "ts_scene_texels": [vp, C.POINTER(vp), C.POINTER(i32), C.POINTER(i32)],
        "ts_scene_set_geometry": [vp, vp, vp, vp, vp, vp],
        "ts_adam_update": [vp, vp, vp, vp, i64, C.POINTER(TsAdam), vp, i32, i32, vp],
        "ts_server_create": [C.POINTER(vp), i32, C.c_size_t, i32, i32],
        "ts_server_destroy": [vp],
        "ts_server_submit": [vp, vp, C.POINTER(TsCamera), C.POINTER(C.c_uint64)],
        "ts_server_wait": [vp, C.c_uint64, vp, i32, C.c_double],
        "ts_server_stats": [vp, C.POINTER(TsServeStats)],
        "ts_server_reset_stats": [vp],
        "ts_measure_fp32_peak": [i32, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "ts_scene_build_atlas2d": [vp, i32, i32, vp],
        "ts_scene_set_sampler": [vp, i32],
        "ts_scene_set_normal_encoding": [vp, i32],
        "ts_scene_envmap": [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(i32)],
        "ts_activate": [i64, vp, vp, vp, vp, vp],
        "ts_activate_backward": [i64, vp, vp, vp, vp, vp, vp, i32, vp],
        "ts_selftest_sort_wait": [i32, vp],
        "ts_debug_fail_alloc": [i64],
        "ts_server_batch_log": [vp, i32, C.POINTER(i32), vp, vp, vp, vp],
        "ts_server_request_bytes": [vp, vp, C.POINTER(TsCamera), C.POINTER(C.c_size_t)],
        "ts_image_loss": [vp, vp, i32, i32, C.c_float, vp, vp, vp],
        "ts_saved_copy_depth": [vp, i32, vp, vp, vp],
        "ts_normal_loss": [vp, i32, C.c_float, vp, vp],
        "ts_upload_indirect": [vp, i32, vp, i32, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.ts_last_error.restype = C.c_char_p
    L.ts_last_error.argtypes = []
    L.ts_version.restype = C.c_char_p
    L.ts_version.argtypes = []
    L.ts_launch_count.restype = C.c_int64
    L.ts_launch_count.argtypes = []
    _lib = L
    return L


def check(status: int, what: str = ""):
    if status != 0:
        msg = lib().ts_last_error().decode(errors="replace")
        raise TexSplatError(f"{what}: {STATUS.get(status, status)}: {msg}")


def launch_count() -> int:
    """Kernels launched by the library so far."""
    return int(lib().ts_launch_count())


def profile_enable(on: bool = True):
    check(lib().ts_profile_enable(1 if on else 0), "ts_profile_enable")


def profile_report() -> dict:
    """{stage: (launches, total_ms)} of the stages timed since the last report."""
    buf = C.create_string_buffer(1 << 16)
    check(lib().ts_profile_report(buf, len(buf)), "ts_profile_report")
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms = line.split()
        out[name] = (int(n), float(ms))
    return out


def measure_fp32_peak(device: int = 0) -> tuple[float, float]:
    """(scalar, paired) FP32 FMA rate of the device in TFLOP/s."""
    a, b = C.c_double(), C.c_double()
    check(lib().ts_measure_fp32_peak(device, C.byref(a), C.byref(b)), "ts_measure_fp32_peak")
    return a.value, b.value
