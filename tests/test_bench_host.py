"""Host logic of bench.py on CPU: the clock summary that decides whether a
run is kept, and the JSON line of the reference arm (the CPU oracle on a
bounded sample) on the small workload."""
import argparse
import contextlib
import io
import json

import bench


def test_clock_summary_median_and_reasons():
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1900, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}


def test_clock_summary_without_samples():
    c = bench.ClockSampler(0)
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_reference_arm_line_on_the_small_workload():
    args = argparse.Namespace(workload="tiny", steps=1, warmup=0, gpus=1, cpu_rows=4)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        assert bench.run_reference(args) == 0
    line = json.loads(out.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "sky-s/s"
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "4 of 200 DM rows" in cb["sample"]
    assert line["config"]["workload"].startswith("tiny: 256 ch")


def test_stream_busy_union():
    import bench
    assert bench.busy_union([]) == (0.0, 0.0)
    # overlapping, nested and disjoint intervals, in any order
    busy, span = bench.busy_union([(5.0, 7.0), (0.0, 2.0), (1.0, 3.0), (1.5, 2.5), (10.0, 11.0)])
    assert busy == 3.0 + 2.0 + 1.0
    assert span == 11.0
