"""bench.py's roofline bookkeeping on CPU: the algorithmic bytes of one
correspondence pass (12 M + 24 N point-to-plane, 12 M + 12 N point-to-point),
the achieved rate over a launch time, the fraction of the measured HBM peak, and
the ncu counters taken only from a profile of the current search-kernel sources."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_roofline_arithmetic():
    peaks = bench.measured_peaks()
    peak = peaks["hbm_gbs"] if peaks and "hbm_gbs" in peaks else 6800.0
    r = bench.roofline_of(500.0, 200_000, 500_000, True, "no_such_workload")
    assert r["algorithmic_bytes_per_launch"] == 12 * 200_000 + 24 * 500_000
    assert r["achieved"] == pytest.approx(14.4e6 / 500e-6 / 1e9)
    assert r["peak"] == peak and r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["traffic"] is None            # no profile for this workload
    r2 = bench.roofline_of(100.0, 80_000, 100_000, False, "no_such_workload")
    assert r2["algorithmic_bytes_per_launch"] == 12 * 80_000 + 12 * 100_000


def test_profile_counters_follow_the_kernel_sources(tmp_path, monkeypatch):
    d = json.loads((bench.ROOT / "profiles" / f"k_nn_{bench.WORKLOAD}.json").read_text())
    r = bench.roofline_of(485.0, 200_000, 500_000, True, bench.WORKLOAD)
    if d["kernel_source_sha256_16"] == bench.step_kernel_hash():
        assert r["traffic"] == d["dram_bytes_per_launch"]
        assert r["issue_active_frac"] == d["issue_active_frac"]
    else:                                   # sources changed since the capture: no counters
        assert r["traffic"] is None
    # a profile taken on other sources is not used
    fake = tmp_path / "profiles"
    fake.mkdir()
    (fake / f"k_nn_{bench.WORKLOAD}.json").write_text(json.dumps(dict(d, kernel_source_sha256_16="0" * 16)))
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    monkeypatch.setattr(bench, "step_kernel_hash", lambda: "1" * 16)
    assert bench.profiled_kernel(bench.WORKLOAD) == {}
