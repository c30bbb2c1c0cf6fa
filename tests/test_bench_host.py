"""Host-side pieces of bench.py that need no GPU: a DRAM-traffic record is
used only while its source hashes match the kernels in the tree (a stale one
makes the bench report traffic as null), its figure is the algorithmic bytes
within a few percent, and the rate arithmetic."""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_current_traffic_records_are_the_algorithmic_bytes():
    for w in ("c2", "c5"):
        rec = bench.traffic_record(w)
        if rec is None:
            pytest.skip(f"the {w} traffic record predates the current kernel sources")
        assert rec["dram_bytes_per_launch"] > 0
        # the capture read the knots once: within 5% of the algorithmic bytes
        assert abs(rec["dram_bytes_per_launch"] / rec["algorithmic_bytes_per_launch"] - 1) < 0.05


def test_a_changed_source_invalidates_the_record(monkeypatch):
    real = bench.sources_sha256
    monkeypatch.setattr(bench, "sources_sha256", lambda files: real(files)[::-1])
    assert bench.traffic_record("c2") is None


def test_record_file_names_its_sources():
    d = json.load(open(os.path.join(ROOT, "profiles", "rollout_traffic.json")))
    for w, rec in d.items():
        assert rec["sources"] == bench.TRAFFIC_SOURCES[w]
        for f in rec["sources"]:
            assert os.path.exists(os.path.join(ROOT, "paper_2001_04931_gb300", "csrc", f))


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(1000, 4, 2.0) == 2000.0


def test_variant_record_keeps_the_roofline_evidence():
    """A variant's record in the default line keeps what its roofline claim
    rests on: the fraction, the kernel's time, its algorithmic work, the DRAM
    traffic figure and, for the tensor-core rollout, the issued MMA work."""
    roof = {"bound": "tensor", "kernel": "k", "achieved": 550.0, "peak": 1912.2, "unit": "TFLOP/s",
            "frac": 0.29, "peak_basis": "measured", "launch_us": 194.0,
            "flops_per_launch": 1.07e11, "mma_flops_per_launch": 1.61e11,
            "traffic": 33712640, "breed_us": 65.0}
    line = {"config": {"workload": "c5"}, "dtype": "bf16", "metric": bench.METRIC, "value": 1.0,
            "unit": bench.UNIT, "steps": 1, "warmup": 3, "ms_per_step": 10.9,
            "ms_per_problem": 10.9, "e2e": {}, "gpu_launches": 120, "clocks": {},
            "roofline": roof, "compare": {"median_speedup": 14.9}}
    out = bench.compact(line)
    for k in ("frac", "launch_us", "flops_per_launch", "mma_flops_per_launch", "traffic"):
        assert out["roofline"][k] == roof[k]
    assert "breed_us" not in out["roofline"]
    assert out["compare"] == line["compare"]
