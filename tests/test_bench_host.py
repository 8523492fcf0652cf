"""Host-side logic of bench.py: multi-rank aggregation (gloo, world size 2, on
CPU), launch counting, the ncu-traffic lookup and the clock summary."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "took" 1 + r seconds for (r + 1) * 100 units
    t, u = bench.aggregate(1.0 + rank, 100.0 * (rank + 1), dist)
    q.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_is_max_time_and_sum_of_units_over_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, u in res:
        assert t == 2.0 and u == 300.0


def test_single_rank_aggregate_passthrough():
    assert bench.aggregate(1.5, 42.0, None) == (1.5, 42.0)


def test_sweep_launch_count():
    # 20000 steps after 200 warm-up: a diagnostic sweep every 100 steps (200 of
    # them, the last step among them) plus one fold kernel each
    assert bench.sweep_launches(200, 20000) == 20000 + 200
    # last step not on the cadence: one extra diagnostic sweep
    assert bench.sweep_launches(0, 150) == 150 + 2
    assert bench.sweep_launches(3, 5) == 5 + 1


def test_profiled_traffic_needs_matching_kernel_hash(tmp_path, monkeypatch):
    prof = tmp_path / "p.md"
    prof.write_text(f"kernel_source_sha256: {bench.kernel_source_hash()}\ndram_bytes_per_launch: 1.5e8\n")
    monkeypatch.setattr(bench, "profile_path", lambda prec, batch=0: str(prof))
    assert bench.profiled_traffic() == 1.5e8
    prof.write_text("kernel_source_sha256: 0000000000000000\ndram_bytes_per_launch: 1.5e8\n")
    assert bench.profiled_traffic() is None


def test_profiled_traffic_is_per_precision(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    h = bench.kernel_source_hash()
    (tmp_path / "profiles" / "sweep_fp32_cavity_2048x1024.md").write_text(
        f"kernel_source_sha256: {h}\ndram_bytes_per_launch: 2.5e8\n")
    assert bench.profiled_traffic("fp32") == 2.5e8
    assert bench.profiled_traffic("bf16sr") is None   # no summary for that precision
    assert bench.profiled_traffic("fp32", 64) is None  # nor for the batch kernel
    (tmp_path / "profiles" / "batch_fp32_64x256x128.md").write_text(
        f"kernel_source_sha256: {h}\ndram_bytes_per_launch: 3.1e8\n")
    assert bench.profiled_traffic("fp32", 64) == 3.1e8


def test_committed_profiles_carry_hash_and_traffic():
    # every committed sweep summary that states a traffic figure also states
    # the kernel source it was taken on
    import glob
    for f in glob.glob(os.path.join(bench.ROOT, "profiles", "sweep_*_cavity_2048x1024.md")):
        text = open(f).read()
        if "dram_bytes_per_launch:" in text:
            assert "kernel_source_sha256:" in text, f


def test_workload_config_states_the_streaming_and_the_l2_footprint():
    # one buffer for every storage type but FP64; the note says whether the
    # buffer a step reads and writes exceeds the 129 MB L2 (FP32: 151 MB) or
    # fits in it (16-bit: 75 MB), and FP64's two buffers (604 MB) exceed it
    fp32, bf16, fp64 = (bench.workload_config(p) for p in ("fp32", "bf16sr", "fp64"))
    assert fp32["streaming"].startswith("one buffer") and bf16["streaming"].startswith("one buffer")
    assert fp64["streaming"] == "two buffers"
    assert fp32["l2"].startswith("inputs larger than L2 (151 MB")
    assert "fit in the 129 MB L2" in bf16["l2"] and "(75 MB" in bf16["l2"]
    assert fp64["l2"].startswith("inputs larger than L2 (2 x 302 MB")


def test_measured_peak_falls_back(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak_gbs() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6784.8}))
    assert bench.measured_peak_gbs() == (6784.8, "measured")


def test_clock_summary_parses_nvidia_smi_csv(tmp_path):
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "c.csv")
    cs.proc = object()  # pretend the sampler ran
    with open(cs.path, "w") as fh:
        fh.write("0, 2070, 2070, 176.5, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        fh.write("0, 1980, 2070, 900.1, 0x4, Not Active, Not Active, Not Active, Active\n")
        fh.write("0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert s["median_of"] == "warm-up and timed region"


def test_clock_summary_of_a_short_region_uses_the_bracket(tmp_path):
    """A timed region shorter than the 100 ms sampling period leaves the loop
    with no sample: the samples taken just before and after it still give a
    clock and the throttle reasons."""
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "c.csv")
    cs.proc = object()
    open(cs.path, "w").close()
    row = "0, 1965, 2070, 700.0, 0x0, Not Active, Not Active, Active, Not Active"
    cs.bracket = [[p.strip() for p in row.split(",")], [p.strip() for p in row.split(",")]]
    s = cs.summary()
    assert s["sm_mhz"] == 1965.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 0
    assert s["reasons"] == ["sw_thermal_slowdown"] and s["bracket_samples"] == 2
    assert s["median_of"].startswith("samples just before")


def test_reference_arm_line(capsys, monkeypatch):
    """--impl reference times the oracle on this host and prints the contract's
    line with the GPU arm's config; ranks other than 0 print nothing."""
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "MLUPS" and line["value"] > 0
    assert line["config"] == bench.workload_config("fp32")
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 3
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert capsys.readouterr().out.strip() == ""
