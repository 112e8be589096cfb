"""bench.py takes per-kernel ncu figures (DRAM traffic, warp-instructions)
from the committed profile summary only when they were recorded on the
current kernel source; otherwise it reports null."""
import bench


def test_profiled_figures_follow_the_source_hash(tmp_path, monkeypatch):
    h = "0123456789abcdef"
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "spmv_fast_hpcg192.md").write_text(
        "# summary\n"
        f"traffic: kernel=k1 source_sha256_16={h} bytes=123\n"
        f"issue: kernel=k1 source_sha256_16={h} warp_inst=456\n"
        "traffic: kernel=k2 source_sha256_16=fedcba9876543210 bytes=789\n"
        f"traffic: kernel=k3 source_sha256_16={h} bytes=not-a-number\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel="": h)
    assert bench.profiled_traffic("k1") == 123.0
    assert bench.profiled("k1", "issue", "warp_inst") == 456.0
    assert bench.profiled_traffic("k2") is None          # taken on another source
    assert bench.profiled_traffic("k3") is None          # unreadable figure
    assert bench.profiled_traffic("k4") is None          # never profiled
    assert bench.profiled("k2", "issue", "warp_inst") is None


def test_no_profile_summary_means_null(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k1") is None


def test_committed_summary_lines_are_well_formed():
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles",
                        "spmv_fast_hpcg192.md")
    n = 0
    with open(path) as f:
        for line in f:
            if line.startswith(("traffic:", "issue:")):
                parts = dict(p.split("=", 1) for p in line.split()[1:])
                assert set(parts) == {"kernel", "source_sha256_16", "bytes" if line.startswith("traffic") else "warp_inst"}
                assert len(parts["source_sha256_16"]) == 16
                float(parts.get("bytes", parts.get("warp_inst")))
                n += 1
    assert n > 0
