"""The benchmark's reference arm (the FP64 oracle on the host cores) runs on
a CPU-only machine and prints one JSON line with the contract's keys."""
import json

import bench


def test_reference_arm_prints_one_contract_line(capsys, monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)

    class Args:
        steps, warmup, cpu_tiles = 1, 0, 3

    assert bench.run_reference(Args) == 0
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"]["workload"] == bench.workload_config(1)["workload"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0
