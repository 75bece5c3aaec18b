"""The bench reports the captured DRAM traffic of the stage kernel only for
the tile shape and kernel sources it was captured with (host logic, CPU)."""
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
    monkeypatch.setitem(bench.NCU_TRAFFIC, "sources", ("a.cuh", "t.h:TABLE"))
    h0 = bench.kernel_sources_sha256()
    (csrc / "t.h").write_text("// header, edited\n#define TABLE(X) \\\n  X(1, 2)\n\nint other;\n")
    assert bench.kernel_sources_sha256() == h0  # outside the block: same kernel
    (csrc / "t.h").write_text("// header\n#define TABLE(X) \\\n  X(1, 3)\n\nint unrelated;\n")
    assert bench.kernel_sources_sha256() != h0  # the table changed
    (csrc / "a.cuh").write_text("kernel code, edited\n")
    assert bench.kernel_sources_sha256() != h0


def test_traffic_is_withheld_for_another_tile_or_changed_sources(monkeypatch):
    cells = 4096 * 4096
    monkeypatch.setitem(bench.NCU_TRAFFIC, "sha256", bench.kernel_sources_sha256())
    got = bench.ncu_traffic(bench.NCU_TRAFFIC["tile"], 2, cells)
    assert got == bench.NCU_TRAFFIC["bytes"][2] / bench.NCU_TRAFFIC["cells"] * cells
    assert bench.ncu_traffic(bench.NCU_TRAFFIC["tile"] + 1, 2, cells) is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, "sha256", "0" * 64)
    assert bench.ncu_traffic(bench.NCU_TRAFFIC["tile"], 2, cells) is None
