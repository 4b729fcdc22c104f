"""Host-side logic of bench.py (no GPU): the algorithmic byte and ALU-op
models of one trace launch, computed from per-ray counter rows
(box tests, triangle tests, intersector calls, texture fetches), and the
rule that profiled per-level traffic is used only while the summary's
source hash and launch configuration match the current ones."""
import numpy as np

import bench

STATS = np.array([[2, 1, 1, 1], [3, 0, 0, 0]], np.uint32)


def test_trace_bytes_by_hand():
    # 2 rays x (32 ray + 16 hit) + 5 boxes x 32 + 1 triangle x 48
    # + 1 call x 4 (geometry id) + 1 fetch x (24 texture coordinates + 4 texel)
    assert bench.trace_bytes(2, STATS, 4, True) == 96 + 160 + 48 + 4 + 28
    assert bench.trace_bytes(2, STATS, 4, False) == 96 + 160 + 48


def test_trace_bytes_procedural_reads_no_texel():
    assert bench.trace_bytes(2, STATS, 0, True) == 96 + 160 + 48 + 4 + 24


def test_trace_load_bytes_leave_out_the_hit_store():
    # 2 rays x 32 ray bytes loaded; the 16-byte hit records are stores
    assert bench.trace_load_bytes(2, STATS, 4, True) == 64 + 160 + 48 + 4 + 28
    assert bench.trace_load_bytes(2, STATS, 0, False) == 64 + 160 + 48


def test_trace_alu_ops_by_hand():
    # 6 per ray, 5 per box test, 7 per triangle test, 1 per call, and the
    # per-lookup work of the intersector (8 alpha texture, 11 procedural)
    assert bench.BOX_TEST_ALU_OPS == 5
    assert bench.trace_alu_ops(2, STATS, bench.ALU_OPS_PER_LOOKUP["alpha_tex"]) == \
        12 + 25 + 7 + 1 + 8
    assert bench.trace_alu_ops(2, STATS, bench.ALU_OPS_PER_LOOKUP["proc_alpha"]) == \
        12 + 25 + 7 + 1 + 11
    assert bench.trace_alu_ops(2, STATS) == 12 + 25 + 7 + 1


def test_adjoint_models_by_hand():
    grad = np.array([True, True, False])
    lit = np.array([True, False, True])
    st = np.array([[2, 1, 1, 1], [3, 0, 0, 0], [1, 0, 0, 0]], np.uint32)
    nbytes, natomics = bench.render_backward_model(3, st, grad, lit)
    trace = 3 * 48 + 32 * 6 + 48 * 1 + 4 * 1 + (24 + 4) * 1 - 16 * 3
    assert nbytes == trace + 2 * (160 + 36) + 48 * 1
    assert natomics == 2 * 9 + 4  # 9 scalar vertex atomics per ray, 4 vector texel atomics
    # from saved hits: 16 B record per ray, 16 B direction + 12 B dL/dc per hit,
    # 148 + 36 B per hit with a gradient, 48 B per lit one
    hit3 = np.array([True, True, False])
    assert bench.render_backward_hits_model(hit3, grad & hit3, lit) == \
        3 * 16 + 2 * (16 + 12) + 2 * (148 + 36) + 48 * 1
    hit = np.array([True, True, True, False])
    tex = np.array([True, True, False, False])
    vis = np.array([True, False, True, True])
    nbytes, natomics = bench.ao_backward_model(hit, tex, vis)
    assert nbytes == 4 * 28 + 3 * 4 + 2 * 100 + 1 * 48 and natomics == 4


def _summary(tmp_path, kernel, digest, config, levels=(11, 22, 33)):
    p = tmp_path / "summary.md"
    p.write_text("# a kernel\n\n    ncu --set full -k regex:k_trace\n\n"
                 f"    kernel: {kernel}\n    kernel_source_hash: {digest}\n"
                 f"    launch_config: {config}\n"
                 f"    l1_bytes_per_launch: {levels[0]}\n    l2_bytes_per_launch: {levels[1]}\n"
                 f"    dram_bytes_per_launch: {levels[2]}\n")
    return str(p)


def test_profiled_levels_need_current_sources_and_config(tmp_path, monkeypatch):
    k = "trace closest alpha (primary)"
    cfg = "block=128 persistent=0 refill=16 stack_regs=4 image_width=1920"
    monkeypatch.setitem(bench.PROFILE_SUMMARIES, k,
                        _summary(tmp_path, k, bench.kernel_source_hash(), cfg))
    assert bench.profiled_levels(k, cfg) == {"l1": 11, "l2": 22, "dram": 33}
    assert bench.profiled_levels(k, cfg.replace("stack_regs=4", "stack_regs=0")) is None
    assert bench.profiled_levels("another kernel", cfg) is None
    monkeypatch.setitem(bench.PROFILE_SUMMARIES, k, _summary(tmp_path, k, "0" * 16, cfg))
    assert bench.profiled_levels(k, cfg) is None
    monkeypatch.setitem(bench.PROFILE_SUMMARIES, k, str(tmp_path / "missing.md"))
    assert bench.profiled_levels(k, cfg) is None


def test_level_fractions():
    out = bench.level_fractions({"l1": 2e9, "l2": 1e9, "dram": 1e8}, 1.0,
                                {"l1": 4000.0, "l2": 2000.0, "dram": 1000.0})
    assert out["l1"]["GBs"] == 2000.0 and out["l1"]["frac"] == 0.5
    assert out["l2"]["frac"] == 0.5 and out["dram"]["frac"] == 0.1
