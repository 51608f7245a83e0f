"""bench.py's profile bookkeeping (no GPU): the source fingerprint ignores comments and blank
lines but not code, and a profile's DRAM traffic is used only while its fingerprint matches."""
import os
import shutil

import bench

FILES = ("kernels.cu", "imrt_internal.cuh", "ptx.cuh", "format.cu", "api.cu")


def copy_tree(tmp_path):
    src = os.path.join(bench.ROOT, "paper_0908_4421_gb300", "csrc")
    dst = tmp_path / "paper_0908_4421_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in FILES:
        shutil.copy(os.path.join(src, f), dst / f)
    (tmp_path / "profiles").mkdir()
    return dst


def test_fingerprint_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    k = csrc / "kernels.cu"
    text = k.read_text()
    k.write_text("// a new comment line\n\n" + text.replace("\n", "  \n", 3) + "\n/* a block\n comment */\n")
    assert bench.kernel_source_hash() == h0
    k.write_text(text + "\nconstexpr int kUnusedProbe = 1;\n")
    assert bench.kernel_source_hash() != h0


def test_profiled_traffic_only_for_the_current_source(tmp_path, monkeypatch):
    copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    prof = tmp_path / "profiles" / "k_forward_w.md"
    assert bench.profiled_traffic("k_forward", "w") is None  # no summary
    prof.write_text(f"source_sha256_16: {bench.kernel_source_hash()}\ntraffic_bytes_per_launch: 12345\n")
    assert bench.profiled_traffic("k_forward", "w") == 12345
    prof.write_text("source_sha256_16: 0123456789abcdef\ntraffic_bytes_per_launch: 12345\n")
    assert bench.profiled_traffic("k_forward", "w") is None  # stale
