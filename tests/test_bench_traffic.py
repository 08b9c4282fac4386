"""bench.py's DRAM traffic figure, on the CPU: it comes from the committed small
one-kernel capture only while the kernel sources hash as they did at the
capture, only for the captured kernel, half and r, and it is scaled by the
bucket's nonzeros; the record's own figures are consistent with its counters
and with bench.py's algorithmic-bytes formula (8 + 4r per nonzero, 8r + 8 per
unit)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _record():
    with open(os.path.join(ROOT, "profiles", "dram_traffic_small.json")) as f:
        return json.load(f)


def test_traffic_scales_with_bucket_nnz_when_sources_match(monkeypatch):
    d = _record()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: d["kernel_source_hash"])
    kernel, half = d["kernel"].split("/")
    assert bench.ncu_traffic(kernel, half, d["r"], 1000) == pytest.approx(d["dram_bytes_per_nnz"] * 1000)
    assert bench.ncu_traffic(kernel, half, d["r"], 37_600_000) == pytest.approx(d["dram_bytes_per_nnz"] * 37_600_000)
    # another half, another r or another kernel has no figure
    assert bench.ncu_traffic(kernel, "W" if half == "F" else "F", d["r"], 1000) is None
    assert bench.ncu_traffic(kernel, half, d["r"] + 1, 1000) is None
    assert bench.ncu_traffic(kernel + "_other", half, d["r"], 1000) is None


def test_traffic_withheld_once_sources_change(monkeypatch):
    d = _record()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    kernel, half = d["kernel"].split("/")
    assert bench.ncu_traffic(kernel, half, d["r"], 1000) is None


def test_hash_covers_every_kernel_source(tmp_path, monkeypatch):
    # a change to any of the files the sweep kernels are built from changes the hash
    csrc = os.path.join(ROOT, "paper_1604_04026_gb300", "csrc")
    names = ("sweep.cu", "common.cuh", "device_util.cuh")
    fake = tmp_path / "paper_1604_04026_gb300" / "csrc"
    fake.mkdir(parents=True)
    for n in names:
        with open(os.path.join(csrc, n), "rb") as f:
            (fake / n).write_bytes(f.read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    assert h0 == bench.kernel_source_hash()
    for n in names:
        original = (fake / n).read_bytes()
        (fake / n).write_bytes(original + b"\n")
        assert bench.kernel_source_hash() != h0, n
        (fake / n).write_bytes(original)
    assert bench.kernel_source_hash() == h0


def test_record_is_self_consistent():
    d = _record()
    per_nnz = (d["dram_bytes_read"] + d["dram_bytes_write"]) / d["bucket_nnz"]
    assert d["dram_bytes_per_nnz"] == pytest.approx(per_nnz, abs=0.01)
    alg = bench.algorithmic_bytes(d["bucket_nnz"], d["bucket_units"], d["r"]) / d["bucket_nnz"]
    assert d["algorithmic_bytes_per_nnz"] == pytest.approx(alg, abs=0.01)
