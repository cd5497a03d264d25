"""Failure detection without a GPU fault: the radix sort's inter-block wait
is bounded; a pass whose predecessor never runs reports TS_ERR_TIMEOUT
through the host, and the device stays usable."""
import time

import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2506_13348_b300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return P


def test_sort_wait_runs_out_and_is_reported(P):
    from paper_2506_13348_b300 import _lib
    t0 = time.time()
    st = _lib.lib().ts_selftest_sort_wait(0, None)
    dt = time.time() - t0
    assert _lib.STATUS[st] == "TS_ERR_TIMEOUT", _lib.lib().ts_last_error()
    assert dt < 30.0
    # the flag was cleared and the context is usable: a render goes through
    scene = sg.make_scene(0, n=256, T=4, seed=0)
    env = sg.make_env(0, cube_res=8, irr_res=4, lut_res=16)
    sc = P.Scene.from_arrays(scene, env)
    out, _ = P.render(sc, sg.look_at_camera((4.0, 0.0, 0.0), 64, 64))
    torch.cuda.synchronize()
    assert torch.isfinite(out).all() and out[..., 3].max().item() > 0.5
