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


def test_clock_summary_keeps_the_samples_inside_the_timed_window():
    """The bench's clock record is taken over the nvidia-smi samples whose
    timestamps fall inside the timed window; a slowdown reason seen only
    outside it is not attributed to the measurement."""
    import datetime
    base = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def line(ms, mhz, hw="Not Active", cap="Not Active"):
        ts = (base + datetime.timedelta(milliseconds=ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2032, 700.00, 0x0, {hw}, Not Active, Not Active, {cap}\n"

    lines = [line(0, 1200, hw="Active"), line(20, 2032), line(40, 2000, cap="Active"), line(60, 2032),
             line(80, 900, hw="Active"), "garbage\n"]
    t0 = (base + datetime.timedelta(milliseconds=10)).timestamp()
    t1 = (base + datetime.timedelta(milliseconds=70)).timestamp()
    c = bench.summarise_clocks(lines, t0, t1)
    assert c["samples"] == 3 and c["samples_total"] == 5
    assert c["sm_mhz"] == 2032.0 and c["sm_max_mhz"] == 2032.0
    assert c["reasons"] == ["sw_power_cap"]
    # no sample inside a window shorter than the interval: all samples count
    c = bench.summarise_clocks(lines, t0, t0 + 0.001)
    assert c["samples"] == 0 and "hw_slowdown" in c["reasons"]


def test_committed_traffic_is_used_only_for_the_profiled_source_and_launch(monkeypatch, tmp_path):
    """A DRAM-traffic figure from the committed ncu summary is reported only
    while the kernel's sources hash to the profiled value and the bench
    launches as many views per launch as the profiled launch covered."""
    import json
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash("raster_bwd")
    (prof / "traffic.json").write_text(json.dumps(
        {"raster_bwd": {"dram_bytes_per_launch": 123, "views_per_launch": 4, "source_sha256": h},
         "raster_fwd": {"dram_bytes_per_launch": 456, "views_per_launch": 4, "source_sha256": "0" * 64}}))
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(prof / "traffic.json"))
    assert bench.read_traffic("raster_bwd", 4) == 123
    assert bench.read_traffic("raster_bwd", 1) is None      # another launch size
    assert bench.read_traffic("raster_fwd", 4) is None      # sources changed since the capture
    assert bench.read_traffic("sort_pairs", 4) is None      # not a profiled kernel
