"""Host-side arithmetic of the benchmark line: the algorithmic bytes behind
the roofline fraction, and the DRAM-traffic record, which is used only while
the kernel sources hash to the value it was captured with."""
import json

import pytest

import bench


def test_algorithmic_bytes_formula():
    # liquid, interface, gas, obstacle cells; s bytes per stored PDF
    counts = (1000, 100, 50, 10)
    for s in (2, 4, 8):
        want = (1000 + 100 + 50 + 10) * 1 + (1000 + 100) * 38 * s + 100 * 37
        assert bench.algorithmic_bytes(counts, s) == pytest.approx(want)


def test_pure_liquid_bytes_match_the_roofline_table():
    # a lattice of liquid cells moves 38 s + 1 bytes per cell (77 B in 16-bit storage)
    n = 1 << 20
    assert bench.algorithmic_bytes((n, 0, 0, 0), 2) / n == pytest.approx(77.0)
    assert bench.algorithmic_bytes((n, 0, 0, 0), 4) / n == pytest.approx(153.0)


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    rec = {"gas_thread:f16s": {"kernel_sha": bench.kernel_sha(), "dram_bytes_per_launch": 123}}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(p))
    assert bench.traffic_per_launch("f16s", "gas_thread") == 123
    assert bench.traffic_per_launch("fp32", "gas_thread") is None
    rec["gas_thread:f16s"]["kernel_sha"] = "0" * 16
    p.write_text(json.dumps(rec))
    assert bench.traffic_per_launch("f16s", "gas_thread") is None
