"""Atlas pack (float32 -> stored bf16 / f16, round to nearest even): the
stored atlas read back through ts_scene_texels equals torch's conversion,
for the vector path and the scalar fallback (source not 16-byte aligned)."""
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return P


class _DevArray:
    """A device pointer seen by torch through the CUDA array interface."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


@pytest.mark.parametrize("store,tdt", [("bf16", torch.bfloat16), ("f16", torch.float16)])
@pytest.mark.parametrize("aligned", [True, False])
def test_stored_atlas_is_the_rounded_master(P, store, tdt, aligned):
    geo = sg.make_scene(0, n=1000, T=4, seed=3)
    n, T = 1000, 4
    g = torch.Generator().manual_seed(5)
    buf = (torch.randn(n * T * T * 8 + 1, generator=g) * 3).cuda()
    tex = buf[: n * T * T * 8] if aligned else buf[1:]
    assert (tex.data_ptr() % 16 == 0) == aligned
    sc = P.Scene(0)
    sc.upload_gaussians(geo["means"], geo["quats"], geo["scales"], geo["opacity"])
    from paper_2506_13348_b300 import _lib
    from paper_2506_13348_b300.api import DTYPES, _ptr
    _lib.check(_lib.lib().ts_upload_atlas(sc.handle, T, 8, DTYPES[store], _ptr(tex), 1, None), "ts_upload_atlas")
    ptr, T2, dt = P.scene_texels(sc)
    assert T2 == T and dt == DTYPES[store]
    stored = torch.as_tensor(_DevArray(ptr, tex.numel(), "<i2"), device="cuda").clone()
    assert torch.equal(stored, tex.to(tdt).view(torch.int16))
