"""The benchmark's host-side parts (no GPU): workload names and the CPU-baseline record."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as W  # noqa: E402


def test_workload_names():
    assert bench.make_workload("syslog-1MiB-100pat").nbytes == W.MiB
    assert bench.make_workload("syslog-8MiB-1000pat").nbytes == 8 * W.MiB
    with pytest.raises(SystemExit):
        bench.make_workload("no-such-workload")


def test_cpu_baseline_record():
    r = bench.cpu_baseline(W.config1(), budget_s=1.0)
    assert r["kind"] == "oracle" and r["unit"] == "Gbit/s" and r["cores"] >= 1 and r["value"] > 0
    assert "best of" in r["sample"]
    # one thread, and on the 1 MiB configuration the naive oracle as well
    assert r["single_thread"]["value"] > 0 and r["naive"]["value"] > 0
    big = bench.cpu_baseline(W.config2(4 * W.MiB), budget_s=1.0)
    assert "naive" not in big and big["single_thread"]["value"] > 0
