"""B300-native textured 2D Gaussian splat renderer (TextureSplat hot path).

The compute path is libtexsplat.so (hand-written sm_103a CUDA behind the C
ABI in include/texsplat.h); this package is its Python binding.
"""
import importlib

from ._lib import TexSplatError, lib  # noqa: F401

_API = ("Scene", "Saved", "render", "render_views", "render_backward", "zero_grads", "l1_loss", "image_loss", "make_camera",
        "split_spec", "TexSplatRender", "Server", "Trainer", "adam_update", "scene_texels", "scene_envmap",
        "activate", "activate_backward")


def __getattr__(name):
    # the binding needs torch; it is imported on first use so that the build
    # script works without it
    if name in _API:
        return getattr(importlib.import_module(".api", __name__), name)
    raise AttributeError(name)
