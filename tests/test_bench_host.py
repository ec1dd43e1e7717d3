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


def test_dpi_workload_sizes():
    w = bench.make_workload("dpi-16MiB-20000sig")
    assert w.nbytes == 16 * W.MiB and w.seg is not None and int(w.seg[-1]) == w.nbytes
    assert w.patterns.n == 20000


def test_profiles_match_the_kernel_sources(tmp_path, monkeypatch):
    """A committed ncu summary is used only while its source hash equals the kernel's; any other hash (a
    summary taken on another revision of the kernel) gives no figure."""
    sha = bench.kernel_sha()
    assert len(sha) == 16
    for wl, kind, key in (("syslog-256MiB-1000pat", "traffic", "traffic_bytes_per_launch"),
                          ("syslog-256MiB-1000pat", "issue", "inst_per_launch"),
                          ("dpi-2GiB-20000sig", "traffic", "traffic_bytes_per_launch")):
        v = bench.profiled_value(wl, kind, key)
        assert v is not None and v > 0, (wl, kind)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "scan_kernel_x_traffic.md").write_text(
        "kernel sources sha256 prefix: 0000000000000000\ntraffic_bytes_per_launch: 123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sha", lambda: sha)
    assert bench.profiled_value("x", "traffic", "traffic_bytes_per_launch") is None
    (tmp_path / "profiles" / "scan_kernel_x_traffic.md").write_text(
        "kernel sources sha256 prefix: %s\ntraffic_bytes_per_launch: 123\n" % sha)
    assert bench.profiled_value("x", "traffic", "traffic_bytes_per_launch") == 123
