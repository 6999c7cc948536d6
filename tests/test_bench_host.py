"""Host logic of bench.py (CPU only): the committed ncu counters count only for the kernel sources
they were measured on, and the reference arm's configuration names the same workload as the
measured one."""
import json

import bench


def test_counters_tied_to_kernel_sources(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"_about": "test", "_kernel_source_hash": h, "k_brick_gather_t": {"dram_bytes_per_launch": 1.0}}
    (prof / "counters.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    got = bench._counters()
    assert got["k_brick_gather_t"]["dram_bytes_per_launch"] == 1.0 and got["source"] == "test"
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)   # the kernels changed since
    assert bench._counters() == {}


def test_reference_arm_config_matches():
    from paper_1304_2017_gb300 import workloads as W
    geom = W.config("c2")
    a, b = bench._config(geom), bench._config(geom, 1)
    assert a == b and a["transducers"] == 23040 and a["samples"] == 1536 and a["grid"] == [256, 256, 256]
