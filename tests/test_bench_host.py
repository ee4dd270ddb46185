"""Host logic of bench.py (no GPU): the roofline's traffic and instruction
counts are read from the committed ncu summary only while its recorded
source hash matches the fused kernel's sources, else they are null."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, digest, dram="123456789", inst="800000000.000000"):
    p = tmp_path / "summary.md"
    p.write_text(
        "# kernel\n\n"
        f"- kernel_sources_sha256: `{digest}`\n"
        f"- dram_bytes_per_launch: `{dram}`\n\n"
        "| metric | value |\n|---|---|\n"
        f"| `smsp__inst_executed.sum` | {inst} inst |\n")
    return str(p)


def test_counts_read_when_the_sources_match(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", _summary(tmp_path, bench.fused_source_digest()))
    assert bench.profiled_traffic() == 123456789.0
    assert bench.profiled_instructions() == 800000000.0


def test_counts_null_for_other_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", _summary(tmp_path, "0" * 64))
    assert bench.profiled_traffic() is None
    assert bench.profiled_instructions() is None


def test_counts_null_without_a_summary(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "missing.md"))
    assert bench.profiled_traffic() is None
    assert bench.profiled_instructions() is None


def test_source_digest_covers_the_fused_kernel_files():
    csrc = os.path.join(ROOT, "paper_2104_12922_gb300", "csrc")
    for f in bench.FUSED_SOURCES:
        assert os.path.exists(os.path.join(csrc, f)), f
    assert "render_fused.cu" in bench.FUSED_SOURCES and "render_common.cuh" in bench.FUSED_SOURCES
