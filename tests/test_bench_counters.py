"""Host logic of bench.py's roofline counters: the DRAM and instruction counts
taken once by ncu are reported only while the trace kernel's source (trace.cu
and every local header it includes) is the one they were taken on."""
import os
import shutil

import pytest

import bench


def _copy_tree(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2208_10006_gb300", "csrc")
    dst = tmp_path / "paper_2208_10006_gb300" / "csrc"
    shutil.copytree(src, dst)
    return dst


def test_hash_is_stable_for_an_identical_tree(tmp_path, monkeypatch):
    h = bench.trace_source_hash()
    _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.trace_source_hash() == h


@pytest.mark.parametrize("name", ["trace.cu", "dfloat.cuh", "geodesic_df.cuh"])
def test_hash_changes_with_the_kernel_or_an_included_header(tmp_path, monkeypatch, name):
    h = bench.trace_source_hash()
    dst = _copy_tree(tmp_path)
    f = dst / name
    assert f.exists(), name
    f.write_bytes(f.read_bytes() + b"\n// edited\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.trace_source_hash() != h


def test_a_header_outside_the_include_graph_does_not_change_the_hash(tmp_path, monkeypatch):
    h = bench.trace_source_hash()
    dst = _copy_tree(tmp_path)
    (dst / "synth_ops.cuh").write_bytes(b"// edited\n")   # not included by trace.cu
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.trace_source_hash() == h


def test_stale_counters_are_reported_as_null(monkeypatch):
    clk = {"sm_mhz": 2070.0}
    monkeypatch.setattr(bench, "TRACE_COUNTERS_SRC", bench.trace_source_hash())
    assert bench.trace_counters_current()
    live = bench.issue_roofline(2.5, clk, 1000)
    assert live is not None and live["warp_inst_per_launch"] == bench.TRACE_WARP_INST
    assert 0.0 < live["frac"] < 1.5
    monkeypatch.setattr(bench, "TRACE_COUNTERS_SRC", "0" * 16)
    assert not bench.trace_counters_current()
    assert bench.issue_roofline(2.5, clk, 1000) is None
    # the counters describe the N = 1000 workload only
    monkeypatch.setattr(bench, "TRACE_COUNTERS_SRC", bench.trace_source_hash())
    assert bench.issue_roofline(2.5, clk, 400) is None
