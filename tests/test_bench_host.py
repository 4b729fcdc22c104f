"""Host-side logic of bench.py (no GPU): the algorithmic byte and ALU-op
models of one trace launch, computed from per-ray counter rows
(box tests, triangle tests, intersector calls, texture fetches), and the
rule that profiled DRAM traffic is used only while the summary's source
hash matches the current kernel sources."""
import numpy as np

import bench

STATS = np.array([[2, 1, 1, 1], [3, 0, 0, 0]], np.uint32)


def test_trace_bytes_by_hand():
    # 2 rays x (32 ray + 16 hit) + 5 boxes x 32 + 1 triangle x 48
    # + 1 call x 4 (geometry id) + 1 fetch x (24 texture coordinates + 4 texel)
    assert bench.trace_bytes(2, STATS, 4, True) == 96 + 160 + 48 + 4 + 28
    assert bench.trace_bytes(2, STATS, 4, False) == 96 + 160 + 48


def test_trace_alu_ops_by_hand():
    # 6 per ray, 11 per box test, 7 per triangle test, 1 per call, 8 per fetch
    assert bench.trace_alu_ops(2, STATS, True) == 12 + 55 + 7 + 1 + 8
    assert bench.trace_alu_ops(2, STATS, False) == 12 + 55 + 7 + 1


def _summary(tmp_path, kernel, digest, traffic):
    p = tmp_path / "summary.md"
    p.write_text("# a kernel\n\n    ncu --set full -k regex:k_trace\n\n"
                 f"    kernel: {kernel}\n    kernel_source_hash: {digest}\n"
                 f"    traffic_bytes_per_launch: {traffic}\n")
    return str(p)


def test_profiled_traffic_needs_the_current_sources(tmp_path, monkeypatch):
    k = "trace closest alpha (primary)"
    monkeypatch.setattr(bench, "PROFILE_SUMMARY",
                        _summary(tmp_path, k, bench.kernel_source_hash(), 1234))
    assert bench.profiled_traffic(k) == 1234
    assert bench.profiled_traffic("another kernel") is None
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", _summary(tmp_path, k, "0" * 16, 1234))
    assert bench.profiled_traffic(k) is None
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "missing.md"))
    assert bench.profiled_traffic(k) is None
