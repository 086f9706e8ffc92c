"""Host logic of bench.py that needs no GPU: the workload table, the DRAM
traffic records (valid only while the step kernel's source is unchanged), the
clock summary's throttle-reason parsing, and the job throughput."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_workload_table_sizes():
    sizes = {"bubble_512x1024": (512, 1024), "bubble_4096x2048": (2048, 4096),
             "bubble_2048x1024": (1024, 2048), "rising_bubble_120x240": (120, 240),
             "rising_bubble_2048x4096": (2048, 4096), "drop_64x64": (64, 64),
             "merging_256x128": (256, 128)}
    for name, (nx, ny) in sizes.items():
        c = bench.make_case(name, "STF1")
        assert (c.nx, c.ny) == (nx, ny), name
        assert c.phi0.shape == (ny, nx)
    assert bench.walls_name(bench.make_case("rising_bubble_120x240", "STF1")) == "x free-slip+y"
    assert bench.walls_name(bench.make_case("bubble_512x1024", "STF1")) == "y"
    assert bench.walls_name(bench.make_case("drop_64x64", "STF1")) == "none"
    with pytest.raises(SystemExit):
        bench.make_case("no_such_workload", "STF1")


def test_traffic_records_follow_the_kernel_source():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    sha = bench.kernel_sha()
    for key, r in rec.items():
        if key.startswith("_"):
            continue
        workload, storage, stage = key.split("/")
        got = bench.traffic_record(workload, storage, stage)
        if r["kernel_sha"] == sha:
            assert got == pytest.approx(r["dram_bytes_per_lup"])
            assert 40.0 < got < 200.0  # bytes per node update: a plausible DRAM figure
            assert os.path.exists(os.path.join(ROOT, r["source"]))
        else:
            assert got is None
    assert bench.traffic_record("no_such_workload", "fp32", "gather") is None


def test_clock_summary_reads_throttle_reasons():
    c = bench.ClockSampler(0)
    c.rows = [["2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active",
               "Not Active"],
              ["1995", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active",
               "Active"],
              ["2070", "2070", "1200.0", "0x0", "Not Active", "Not Active", "Not Active",
               "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_job_throughput_and_algorithmic_bytes():
    # whole-job GLUPS: nodes x steps x ranks / seconds
    assert bench.job_glups(1, 524288, 200, 0.0056) == pytest.approx(524288 * 200 / 0.0056 / 1e9)
    assert bench.job_glups(4, 1000, 10, 1.0) == pytest.approx(4e4 / 1e9)
    # 18 populations read and written plus phi u read and written, float32;
    # 16-bit storage: 17 populations in 2 bytes, h_0 and phi u in 4
    assert bench.BYTES_PER_LUP["fp32"] == (18 * 2 + 2 * 2) * 4
    assert bench.BYTES_PER_LUP["fp16"] == 17 * 2 * 2 + (1 * 2 + 2 * 2) * 4
    assert bench.L2_FLUSH_BYTES > 129e6


def test_pattern_failures_stay_in_their_entry(monkeypatch):
    """A failing side measurement of the default line is reported in its
    own entry; the others and the plain value are kept."""
    def boom(*a, **k):
        raise RuntimeError("out of memory")
    monkeypatch.setattr(bench, "measure_storage",
                        lambda args, case, dev, st, steps: {"value": 2.0, "unit": "GLUPS"})
    monkeypatch.setattr(bench, "measure_batch", boom)
    monkeypatch.setattr(bench, "measure_adjoint",
                        lambda a, consistency=True: {"value": 13.0,
                                                     "adjoint": {"cost_over_forward": 5.0}})

    class Args:
        steps = 3
    out = bench.measure_patterns(Args(), None, None, 1.0)
    assert out["plain_fp32"]["value"] == 1.0
    assert out["fp16"]["vs_plain"] == 2.0 and out["bf16"]["value"] == 2.0
    assert out["batch256"] == {"error": "RuntimeError: out of memory"}
    assert out["adjoint_shear"]["cost_over_forward"] == 5.0
