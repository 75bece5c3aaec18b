"""The bench reports the ncu counters of the stage kernel (DRAM traffic,
executed instructions, issue share) only for the tile shape and kernel
sources they were captured with (host logic, CPU)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_hash_covers_only_the_named_block_of_the_shape_header(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2301_12010_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cuh").write_text("kernel code\n")
    (csrc / "t.h").write_text("// header\n#define TABLE(X) \\\n  X(1, 2)\n\nint unrelated;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.NCU_CAPTURE, "sources", ("a.cuh", "t.h:TABLE"))
    h0 = bench.kernel_sources_sha256()
    (csrc / "t.h").write_text("// header, edited\n#define TABLE(X) \\\n  X(1, 2)\n\nint other;\n")
    assert bench.kernel_sources_sha256() == h0  # outside the block: same kernel
    (csrc / "t.h").write_text("// header\n#define TABLE(X) \\\n  X(1, 3)\n\nint unrelated;\n")
    assert bench.kernel_sources_sha256() != h0  # the table changed
    (csrc / "a.cuh").write_text("kernel code, edited\n")
    assert bench.kernel_sources_sha256() != h0


def test_counters_are_withheld_for_another_tile_or_changed_sources(monkeypatch):
    cells = 4096 * 4096
    monkeypatch.setitem(bench.NCU_CAPTURE, "sha256", bench.kernel_sources_sha256())
    monkeypatch.setitem(bench.NCU_CAPTURE, "cells", 2048 * 2048)
    monkeypatch.setitem(bench.NCU_CAPTURE, "dram_bytes", {1: 1.0e8, 2: 1.5e8, 3: 1.4e8})
    monkeypatch.setitem(bench.NCU_CAPTURE, "thread_inst_per_cell", {1: 500.0, 2: 510.0, 3: 511.0})
    monkeypatch.setitem(bench.NCU_CAPTURE, "issue_active_pct", {1: 60.0, 2: 61.0, 3: 62.0})
    got = bench.ncu_counters(bench.NCU_CAPTURE["tile"], 2, cells)
    assert got["dram_bytes"] == 1.5e8 * 4  # scaled by cells
    assert got["thread_inst_per_cell"] == 510.0 and got["issue_active_pct"] == 61.0
    assert bench.ncu_counters(bench.NCU_CAPTURE["tile"] + 1, 2, cells) is None
    monkeypatch.setitem(bench.NCU_CAPTURE, "sha256", "0" * 64)
    assert bench.ncu_counters(bench.NCU_CAPTURE["tile"], 2, cells) is None
    monkeypatch.setitem(bench.NCU_CAPTURE, "sha256", None)
    assert bench.ncu_counters(bench.NCU_CAPTURE["tile"], 2, cells) is None


def test_issue_ceiling_from_the_captured_instructions(monkeypatch):
    # 152 SMs x 4 schedulers x 32 lanes x clock over the thread instructions
    # of the three stages; withheld when the kernel changed since the capture
    monkeypatch.setitem(bench.NCU_CAPTURE, "sha256", bench.kernel_sources_sha256())
    monkeypatch.setitem(bench.NCU_CAPTURE, "thread_inst_per_cell", {1: 500.0, 2: 600.0, 3: 700.0})
    got = bench.issue_ceiling(1.0e10, {"sm_mhz": 2000.0})
    assert got["thread_inst_per_cell_update"] == 1800.0
    assert abs(got["value"] - 152 * 4 * 32 * 2.0e9 / 1800.0) <= 1e-6 * got["value"]
    assert abs(got["frac"] - 1.0e10 / got["value"]) <= 1e-12
    monkeypatch.setitem(bench.NCU_CAPTURE, "sha256", "0" * 64)
    assert bench.issue_ceiling(1.0e10, {"sm_mhz": 2000.0}) is None
