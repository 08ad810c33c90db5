"""bench.py's DRAM-traffic lookup (roofline.traffic): a committed ncu summary counts only for the
batch size it was taken at and only while every kernel's source file still hashes to the value the
summary records (host only, against a temporary profile directory)."""
import hashlib
import os

import bench


def _setup(tmp_path, monkeypatch, batch=256):
    src = tmp_path / "k.cu"
    src.write_text("kernel source\n")
    other = tmp_path / "g.cu"
    other.write_text("another kernel\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()
    hg = hashlib.sha256(other.read_bytes()).hexdigest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic_w.txt").write_text(
        "# DRAM bytes per launch\n"
        f"# batch {batch}\n"
        "# kernel bytes_per_launch source sha256(source)\n"
        f"k_a 1000 k.cu {h}\n"
        f"k_b 234 k.cu {h}\n"
        f"k_c 50 g.cu {hg}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return src, other


def test_sum_over_the_launchers_kernels(tmp_path, monkeypatch):
    _setup(tmp_path, monkeypatch)
    assert bench.measured_traffic(["k_a", "k_b"], "w", 256) == 1234
    assert bench.measured_traffic(["k_c"], "w", 256) == 50


def test_none_for_another_batch_a_missing_kernel_or_workload(tmp_path, monkeypatch):
    _setup(tmp_path, monkeypatch)
    assert bench.measured_traffic(["k_a"], "w", 128) is None
    assert bench.measured_traffic(["k_a", "k_missing"], "w", 256) is None
    assert bench.measured_traffic(["k_a"], "other", 256) is None


def test_a_changed_source_voids_its_kernels_only(tmp_path, monkeypatch):
    src, _ = _setup(tmp_path, monkeypatch)
    src.write_text("kernel source, changed\n")
    assert bench.measured_traffic(["k_a"], "w", 256) is None
    assert bench.measured_traffic(["k_a", "k_c"], "w", 256) is None
    assert bench.measured_traffic(["k_c"], "w", 256) == 50
    os.remove(src)
    assert bench.measured_traffic(["k_b"], "w", 256) is None
