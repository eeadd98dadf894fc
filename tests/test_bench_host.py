"""The benchmark's host-side bookkeeping (CPU): clock-sample parsing and the rule
that an ncu figure is reported only while the kernel sources match the profile."""
import os
import shutil

import pytest

import bench


def test_clock_summary_parses_samples_and_reasons():
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 2070, 2070, 800.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["0, 1500, 2070, 900.0, 0x0, Active, Not Active, Active, Not Active"]
    assert bench.ClockSampler.summary(c)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["reasons"] == ["no samples"]


def test_profile_figures_only_for_the_profiled_sources(tmp_path):
    """A summary stamped with the current sources gives its figures; one stamped
    with other sources, or a missing one, gives none."""
    sha = bench.kernel_source_sha256()
    text = ("traffic_bytes_per_launch: 77.35e6\nl2_read_bytes_per_launch: 1.802e9\n"
            "l2_throughput_frac: 0.151\nkernel_source_sha256: " + sha + "\n")
    fresh = tmp_path / "fresh.md"
    fresh.write_text(text)
    assert bench.profile_traffic(str(fresh)) == 77.35e6
    assert bench.profile_value("l2_read_bytes_per_launch", str(fresh)) == 1.802e9
    assert bench.profile_value("l2_throughput_frac", str(fresh)) == 0.151
    stale = tmp_path / "stale.md"
    stale.write_text(text.replace(sha, "0" * 64))
    assert bench.profile_traffic(str(stale)) is None
    assert bench.profile_value("l2_throughput_frac", str(stale)) is None
    assert bench.profile_traffic(str(tmp_path / "missing.md")) is None
    # the committed summaries carry the figures the bench reads
    for name in ("bfs_dcsbm16384.md", "bfs_sbm262144.md"):
        committed = open(os.path.join(bench.ROOT, "profiles", name)).read()
        for key in ("traffic_bytes_per_launch", "kernel_source_sha256"):
            assert key + ":" in committed, (name, key)


def test_kernel_source_hash_follows_the_sources(tmp_path, monkeypatch):
    """Any edit of the BFS sources changes the hash (and so retires the profile's
    figures)."""
    sha = bench.kernel_source_sha256()
    assert len(sha) == 64 and sha == bench.kernel_source_sha256()
    copy = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "paper_2305_14641_gb300", "csrc"), copy / "paper_2305_14641_gb300" / "csrc")
    csrc = copy / "paper_2305_14641_gb300" / "csrc"
    monkeypatch.setattr(bench, "KERNEL_SRC", [str(csrc / os.path.basename(p)) for p in bench.KERNEL_SRC])
    assert bench.kernel_source_sha256() == sha
    src = csrc / "bfs.cu"
    src.write_text(src.read_text() + "\n// edited\n")
    assert bench.kernel_source_sha256() != sha
