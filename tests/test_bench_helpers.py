"""Host-side helpers of the benchmark: the per-launch DRAM traffic is read from a committed
ncu summary only while the kernel's source file is unchanged since the capture, and the
algorithmic byte counts follow their stated formulas."""
import hashlib
import os

import bench


def test_traffic_is_null_for_a_changed_or_unknown_kernel(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_1512_05820_gb300", "csrc", bench.KERNEL_SOURCE["k_update_v4"])
    digest = hashlib.sha1(open(src, "rb").read()).hexdigest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.txt").write_text(f"traffic_bytes_per_launch k_update_v4 mixed 22 1234 {digest[:12]}\n"
                                f"traffic_bytes_per_launch k_dir_v4 mixed 22 999 {'0' * 12}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the summary's key matches the current source only through the real csrc path
    os.symlink(os.path.join(os.path.dirname(src), ".."), tmp_path / "paper_1512_05820_gb300")
    assert bench.traffic_from_profiles("k_update_v4", "mixed", 22) == 1234.0
    assert bench.traffic_from_profiles("k_update_v4", "mixed", 8) is None      # other width
    assert bench.traffic_from_profiles("k_update_v4", "fp64", 22) is None      # other precision
    assert bench.traffic_from_profiles("k_dir_v4", "mixed", 22) is None        # stale source key
    assert bench.traffic_from_profiles("no_such_kernel", "mixed", 22) is None


def test_spmv_bytes():
    n, nnz = 1000, 7000
    assert bench.b_spmv(n, nnz) == 12 * nnz + 4 * (n + 1) + 16 * n
    assert bench.b_spmv(n, nnz, fp32=True) == 8 * nnz + 4 * (n + 1) + 8 * n
