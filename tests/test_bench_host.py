"""Host-side checks of bench.py's contract that need no GPU: the reference
arm (the CPU oracle) prints one JSON line with the required keys, the CPU
baseline leg describes its sample, and committed ncu figures are tied to the
sources of the kernel they were taken on."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "tiny_256", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "workload" in d["config"]


def test_cpu_baseline_whole_small_workload():
    import bench
    scene, _ = bench.make_scene("tiny_256")
    cb = bench.cpu_baseline(scene)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["unit"] == bench.UNIT
    assert cb["sample"].startswith("the whole workload (8000 segments")


def test_traffic_record_follows_kernel_sources(tmp_path, monkeypatch):
    import bench
    h = bench.kernel_src_hash("raster_kernel")
    hr = bench.kernel_src_hash("resolve_kernel")
    assert h == bench.kernel_src_hash("raster_kernel") and h != hr
    rec = {"single_1080p": {"raster_kernel": {"dram_bytes_per_launch": 123.0, "red_sectors": 90.0,
                                              "warp_inst_per_launch": 10.0, "fp32_flop_per_launch": 4.0,
                                              "src_hash": h},
                            "resolve_kernel": {"dram_bytes_per_launch": 456.0, "src_hash": "stale"},
                            "resolve_tiles_kernel": {"dram_bytes_per_launch": 1.0, "warp_inst_per_launch": 2.0,
                                                     "src_hash": hr}}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.ncu_traffic("raster_kernel", "single_1080p") == 123.0
    assert bench.ncu_entry("raster_kernel", "single_1080p")["red_sectors"] == 90.0
    assert bench.ncu_traffic("resolve_kernel", "single_1080p") is None     # taken on other sources
    assert bench.ncu_traffic("raster_kernel", "crowd_4k") is None          # other workload
    # a pass's counters need every kernel's record on the current sources
    assert bench.ncu_phase(("raster_kernel",), "single_1080p")["warp_inst_per_launch"] == 10.0
    assert bench.ncu_phase(("resolve_tiles_kernel", "resolve_kernel"), "single_1080p") is None
    v = bench.alu_views(bench.ncu_phase(("raster_kernel",), "single_1080p"), 1e-6, {"sm_mhz": 2000.0}, 148)
    assert abs(v["issue"]["frac"] - 10.0 / 1e-6 / (148 * 4 * 2e9)) < 1e-12
    assert abs(v["fp32"]["frac"] - 4.0 / 1e-6 / (148 * 128 * 2 * 2e9)) < 1e-12


def test_forced_tuning_skips_the_autotuner():
    """--tuning k=v,... sets those hm_tuning fields (the binned rasterizer
    here) without timing anything; launches per frame follow the raster mode."""
    import argparse
    import bench
    from paper_2607_04230_b300 import hm
    saved = hm.get_tuning()
    try:
        args = argparse.Namespace(tuning="raster_bin_w=32,raster_bin_h=16,raster_bin_chunk=1024", no_autotune=False)
        res = bench.choose_tuning(args, None, None, 0, n=1)
        assert res["forced"] and res["table"] == [] and res["ms"] is None
        assert (res["tuning"]["raster_bin_w"], res["tuning"]["raster_bin_h"], res["tuning"]["raster_bin_chunk"]) == \
            (32, 16, 1024)
        assert bench.launches_per_frame() == bench.LAUNCHES_PER_FRAME + 3
        hm.set_tuning(raster_bin_w=0, raster_bin_h=0, raster_bin_chunk=0)
        assert bench.launches_per_frame() == bench.LAUNCHES_PER_FRAME
        assert bench.choose_tuning(argparse.Namespace(tuning="", no_autotune=True), None, None, 0, n=1) is None
    finally:
        hm.set_tuning(**saved)
