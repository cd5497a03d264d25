"""Seeded synthetic inputs for the textured-2DGS renderer and its oracle.

This package holds input generation only: splat clouds, texel arrays,
cameras, environment cubemaps, the split-sum BRDF table and target images.
It contains none of the rendering arithmetic (no intersection, filtering,
compositing or shading), so both the CUDA path and the CPU oracle can take
their inputs from here without sharing any method code.

Every array is float32 unless stated; the renderer and the oracle read the
same arrays.
"""
from .scenes import (  # noqa: F401
    CONFIGS,
    make_scene,
    scene_config,
    look_at_camera,
    fibonacci_cameras,
    random_sphere_cameras,
    make_env,
    constant_env,
    brdf_lut,
    make_target,
    random_unit_quats,
    frames_to_quats,
    slice_scene,
)
