"""The bench's guard on recorded ncu traffic (CPU): the record applies only to
the projector sources it was taken on (comments and whitespace aside) and to
its own workload."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

FILES = ("forward.cu", "backward.cu", "bodies.cuh", "epilogue.cuh", "petvr_internal.cuh")


def _tree(tmp_path):
    csrc = tmp_path / "paper_2106_03172_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in FILES:
        shutil.copy(os.path.join(ROOT, "paper_2106_03172_gb300", "csrc", name), csrc / name)
    (tmp_path / "profiles").mkdir()
    return csrc


def test_digest_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.kernel_source_digest()
    f = csrc / "forward.cu"
    f.write_text(f.read_text() + "\n// a comment\n/* and a\n   block comment */\n\n")
    assert bench.kernel_source_digest() == base
    f.write_text(f.read_text() + "static const int kAddedForTheTest = 1;\n")
    assert bench.kernel_source_digest() != base


def test_traffic_record_needs_matching_sources_and_workload(tmp_path, monkeypatch):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = tmp_path / "profiles" / "roofline_traffic.txt"
    rec.write_text("# a note: with a colon\nworkload: c256\n"
                   f"source_sha256: {bench.kernel_source_digest()}\nkind1_dram_bytes_per_launch: 1234\n")
    assert bench.dram_traffic_record(1, "c256") == 1234.0
    assert bench.dram_traffic_record(0, "c256") is None          # kind not recorded
    assert bench.dram_traffic_record(1, "c64") is None           # another workload
    rec.write_text(rec.read_text().replace("source_sha256: ", "source_sha256: 0"))
    assert bench.dram_traffic_record(1, "c256") is None          # other sources

