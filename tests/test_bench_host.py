"""Host-side helpers of bench.py (no GPU): the code-only hash that keys the committed ncu traffic
figures to the kernel sources they were captured on, the lookup of those figures, and the
fallback of the measured peaks."""
import json
import os
import shutil

import bench


def _tree(tmp_path):
    """A copy of the kernel sources under a temporary root, for bench's path helpers."""
    src = os.path.join(bench.ROOT, "paper_2306_17263_gb300", "csrc")
    dst = tmp_path / "paper_2306_17263_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("k_tiled.cu", "k_tiled.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    (tmp_path / "profiles").mkdir()
    return dst


def test_code_only_drops_comments_and_blank_lines():
    text = "int a; // trailing\n\n/* block\n   comment */ int b;\n   // whole line\nint c;\n"
    assert bench._code_only(text) == "int a;\n int b;\nint c;"


def test_hash_ignores_comment_edits_and_follows_code_edits(tmp_path, monkeypatch):
    csrc = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_hash("curl32")
    assert h0 == bench.kernel_sources_hash("solve32")  # same files define both kinds
    p = csrc / "k_tiled.cu"
    p.write_text(p.read_text() + "\n// a note added later\n/* and a block */\n")
    assert bench.kernel_sources_hash("curl32") == h0
    p.write_text(p.read_text() + "\nstatic int added_symbol = 0;\n")
    assert bench.kernel_sources_hash("curl32") != h0


def test_traffic_is_reported_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    csrc = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    path = tmp_path / "profiles" / "traffic.json"
    entry = {"sources_sha": bench.kernel_sources_hash("solve32"), "dram_bytes_per_launch": 123.0}
    path.write_text(json.dumps({"solve32": entry}))
    assert bench.ncu_traffic("solve32") == 123.0
    assert bench.ncu_traffic("curl32") is None  # no entry
    p = csrc / "k_tiled.cu"
    p.write_text(p.read_text() + "\nstatic int changed = 1;\n")
    assert bench.ncu_traffic("solve32") is None  # the kernel changed since the capture
    path.write_text("{ not json")
    assert bench.ncu_traffic("solve32") is None


def test_measured_peaks_fall_back_without_the_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    hbm, src = bench.measured_peaks()
    assert src == "fallback" and hbm == bench.FALLBACK_HBM_GBS
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6000.5, "bf16_tflops": 1800}))
    assert bench.measured_peaks() == (6000.5, "measured")
    assert bench.bf16_peak() == 1800.0
