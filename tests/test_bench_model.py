"""The benchmark's byte counts are the paper's traffic model (Section 4:
Eq. (3) plus x read once and y written once), and its recorded DRAM
counters are reported only for the kernel source they were taken on.
Runs on CPU."""
import json
import os

import numpy as np

import bench
import workloads as W
from oracle import traffic as T


def test_spmv_bytes_is_the_traffic_model():
    for n, nnz in ((4096, 20224), (2_097_152, 14_581_760), (4_096_000, 109_215_352)):
        for ib in (1, 2, 4):
            for vb, xb in ((8, 8), (4, 4), (2, 4)):
                want = T.matrix_traffic(n, nnz, 4, ib, vb) + n * xb + n * xb
                assert bench.spmv_bytes(n, nnz, ib, vb, xb) == want
        # with matching value and vector types this is the oracle's SpMV traffic
        assert bench.spmv_bytes(n, nnz, 2, 8, 8) == T.spmv_traffic(n, n, nnz, 4, 2, 8)


def test_headline_workload_sizes_and_bytes():
    rp, col, _ = W.laplace3d_7pt(bench.GRID)
    n, nnz = len(rp) - 1, len(col)
    assert (n, nnz) == (2_097_152, 14_581_760)
    assert int(np.max(np.abs(col.astype(np.int64) - np.repeat(np.arange(n), np.diff(rp))))) \
        == bench.GRID * bench.GRID
    b16 = bench.spmv_bytes(n, nnz, 2, 8, 8)
    b32 = bench.spmv_bytes(n, nnz, 4, 8, 8)
    assert b16 == 187_760_644
    # model speedup of DA-CSR-16 over CSR-32 on this matrix (Eq. (1))
    assert abs(T.performance_ratio(b16, b32) - 1.1553) < 1e-4
    # the four copies the timed steps cycle through exceed the 126 MB L2
    assert bench.NCOPY * b16 > 3 * 126e6


def test_recorded_traffic_only_for_the_profiled_source(monkeypatch):
    path = os.path.join(bench.ROOT, "profiles", "spmv_dacsr16_f64_laplace3d_128.json")
    with open(path) as f:
        rec = json.load(f)
    assert rec["dram_bytes_per_launch"] == \
        rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]
    assert rec["algorithmic_bytes_per_launch"] == bench.spmv_bytes(2_097_152, 14_581_760, 2, 8, 8)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["kernel_source_hash"])
    assert bench.recorded_traffic() == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic() is None


def test_kernel_source_hash_ignores_comments(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2307_06305_gb300", "csrc")
    names = ("spmv_kernel.cuh", "spmv_launch.cuh", "spmv.cu", "damn_common.cuh")
    for name in names:
        with open(os.path.join(src, name)) as f:
            (tmp_path / name).write_text(f.read())
    fake_root = tmp_path / "root"
    (fake_root / "paper_2307_06305_gb300").mkdir(parents=True)
    (fake_root / "paper_2307_06305_gb300" / "csrc").symlink_to(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    h0 = bench.kernel_source_hash()
    assert h0 == bench.kernel_source_hash()
    p = tmp_path / "spmv.cu"
    p.write_text("// a new comment line\n" + p.read_text() + "\n/* block\n comment */\n\n")
    assert bench.kernel_source_hash() == h0
    p.write_text(p.read_text() + "static int changed_code = 1;\n")
    assert bench.kernel_source_hash() != h0


def test_profile_case_names():
    """The --case names the committed ncu summaries use are accepted, and
    malformed ones are refused before any GPU work."""
    import argparse
    import pytest
    ok = ["laplace3d_128", "laplace3d_128_values", "laplace3d_128_dacoo16",
          "stencil27_160_rows_long", "cg_ir_160_bf16", "batch512_f64_k1",
          "batch512_f64_k1_streamed_e2", "batch512_f64_k1_passes_e2", "batch512_f32_k16_streamed",
          "banded_1e6_h1000_band_da16", "banded_1e5_h30000_rows_long_csr32"]
    for name in ok:
        assert bench.profile_case(name) == name
    bad = ["batch512_f64_k0_streamed", "batch512_f64_k65_passes", "batch512_f16_k1_passes",
           "batch512_f64_k1_streamed_e3", "banded_1e6_h1000_band_da8", "banded_1e6_1000_band_da16",
           "laplace3d_64"]
    for name in bad:
        with pytest.raises(argparse.ArgumentTypeError):
            bench.profile_case(name)
