"""Pins of the traffic model (Eq. (1), Eq. (3), Section 4, Fig. 3) against the
numbers the paper prints."""
from fractions import Fraction

import pytest

from oracle import traffic as T


def test_bump2911_example(golden):
    g = golden("bump2911_traffic.txt")
    n, nnz = int(g["nrows"][0]), int(g["nnz"][0])
    mib = T.MIB
    rowptr = T.matrix_traffic(n, 0, 4, 0, 0)
    col32 = nnz * 4
    col16 = nnz * 2
    v64, v32 = nnz * 8, nnz * 4
    # (nrows+1) * |oindex| with oindex int32
    assert rowptr == (n + 1) * 4
    assert round(rowptr / mib) == int(g["mib_rowptr_int32"][0])
    assert round(col32 / mib) == int(g["mib_colids_int32"][0])
    assert round(col16 / mib) == int(g["mib_colids_int16"][0])
    assert round(v64 / mib) == int(g["mib_values_float64"][0])
    assert round(v32 / mib) == int(g["mib_values_float32"][0])
    # bytes of bookkeeping per entry: 4.09 -> 2.09
    assert round(float(T.bytes_per_entry(n, nnz, 4, 4)), 2) == float(g["bytes_per_nnz_csr32"][0])
    assert round(float(T.bytes_per_entry(n, nnz, 4, 2)), 2) == float(g["bytes_per_nnz_dacsr16"][0])
    # the paper's percentages, from its rounded MiB figures
    r = lambda a, b: round(100 * (1 - a / b), 1)
    assert r(11 + 244, 11 + 487) == float(g["reduction_bookkeeping_pct"][0])
    assert r(11 + 244 + 975, 11 + 487 + 975) == float(g["reduction_total_float64_pct"][0])
    assert r(11 + 244 + 487, 11 + 487 + 487) == float(g["reduction_total_float32_pct"][0])
    # the same reductions from Eq. (3) with exact sizes agree to 0.1 %
    full = lambda i, s: T.matrix_traffic(n, nnz, 4, i, s)
    assert abs(100 * (1 - full(2, 8) / full(4, 8)) - 16.5) < 0.1
    assert abs(100 * (1 - full(2, 4) / full(4, 4)) - 24.7) < 0.1
    assert abs(100 * (1 - (full(2, 0)) / full(4, 0)) - 48.8) < 0.15
    # |oindex| = 0 approximations: 1/6 and 1/4
    assert 1 - T.approx_traffic_ratio("int32", "float64", "int16", "float64") == Fraction(g["approx_reduction_float64"][0])
    assert 1 - T.approx_traffic_ratio("int32", "float32", "int16", "float32") == Fraction(g["approx_reduction_float32"][0])


def test_fig3_lattice(golden_rows):
    rows = golden_rows("fig3_traffic_ratios.txt")
    assert len(rows) == 20
    for fi, fs, ti, ts, ratio in rows:
        assert T.approx_traffic_ratio(fi, fs, ti, ts) == Fraction(ratio), (fi, fs, ti, ts)


def test_predicted_speedups(golden_rows):
    for fi, fs, ti, ts, sp in golden_rows("predicted_speedups.txt"):
        assert T.predicted_speedup(fi, fs, ti, ts) == Fraction(sp)


def test_eq1_memory_bound():
    # Eq. (1): half the traffic -> twice the performance
    assert T.performance_ratio(100, 200) == 2
    assert T.performance_ratio(12, 10) == Fraction(5, 6)


def test_work_and_metrics():
    # Section 4: W = 2 nnz + 2 nrows
    assert T.spmv_work(20224, 4096) == 2 * 20224 + 2 * 4096
    assert T.relative_performance(12, 10) == Fraction(6, 5)
    # relative throughput is the relative performance scaled by the traffic ratio
    assert T.relative_throughput(10, 12, 12, 10) == Fraction(10, 12) * Fraction(12, 10)


def test_spmv_traffic_counts_x_and_y():
    n, nnz = 4096, 20224
    a = T.matrix_traffic(n, nnz, 4, 2, 8)
    assert T.spmv_traffic(n, n, nnz, 4, 2, 8) == a + 2 * 8 * n
    assert T.spmv_traffic(n, n, nnz, 4, 2, 8, beta_nonzero=True) == a + 3 * 8 * n
    # 7-point Laplacian on 128^3, beta = 0: DA16 187.8 MB, CSR32 216.9 MB (decimal MB)
    n3, nnz3 = 128 ** 3, 7 * 128 ** 3 - 6 * 128 ** 2
    assert abs(T.spmv_traffic(n3, n3, nnz3, 4, 2, 8) / 1e6 - 187.8) < 0.1
    assert abs(T.spmv_traffic(n3, n3, nnz3, 4, 4, 8) / 1e6 - 216.9) < 0.1
