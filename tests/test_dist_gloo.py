"""Host logic of the multi-rank bench (replicas: no collective on the data
path, the job time is the slowest rank's) on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    ms = bench.max_over_ranks(10.0 + 5.0 * r, dist, "cpu")
    views = bench.rank_views(r, 4)
    gathered = [None] * w
    dist.all_gather_object(gathered, views)
    out[r] = (ms, bench.aggregate_value(w, 3, ms), gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_render_different_views():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, value, views = res[r]
        assert ms == 15.0  # max over ranks, the same on every rank
        assert value == pytest.approx(world * 3 * bench.RES * bench.RES / 1e6 / 0.015)
        assert set(views[0]).isdisjoint(views[1])


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, cpu_tiles = 1, 0, 3

    assert bench.run_reference(Args) == 0  # returns at once, no work


def test_single_rank_defaults():
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.rank_views(0, 3) == [0, 1, 2]
    assert torch.tensor(bench.aggregate_value(1, 2, 1000.0)).item() == pytest.approx(2 * 0.64)
