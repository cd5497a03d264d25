"""The C-ABI library loads and exports every entry point include/texsplat.h
declares (CPU: no compute call is made)."""
import os
import re

import paper_2506_13348_b300 as P
from paper_2506_13348_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "texsplat.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"\b(ts_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    syms = declared_symbols()
    for name in ("ts_create_scene", "ts_upload_gaussians", "ts_upload_atlas", "ts_upload_envmap",
                 "ts_render", "ts_render_backward"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    L = P.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name
    assert set(declared_symbols()) <= set(_lib.EXPORTED) | set(declared_symbols())
    assert b"sm_103a" in L.ts_version()


def test_error_path_without_gpu_or_bad_args():
    import ctypes as C
    L = P.lib()
    # a NULL output handle is rejected before any device work
    assert L.ts_create_scene(None, 0) == 1
    assert L.ts_last_error()
    assert L.ts_render(None, None, None, None, None) != 0
    # null outputs of the FP32 rate probe are rejected before any device work
    assert L.ts_measure_fp32_peak(0, None, None) == 1
