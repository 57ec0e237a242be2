"""Traffic and performance model of the paper (Section 1, Section 2 and
Section 4).  Test infrastructure only (see ``oracle/__init__.py``).

All functions return exact ``fractions.Fraction`` values where the inputs are
integers, so that the tests can compare against the paper's printed ratios
without rounding.
"""
from __future__ import annotations

from fractions import Fraction

MIB = 1 << 20

# Byte sizes of the scalar and index types drawn in Fig. 3.
SCALAR_BYTES = {"float64": 8, "float32": 4, "float16": 2, "float8": 1}
INDEX_BYTES = {"int32": 4, "int16": 2, "int8": 1, "dense": 0}


def performance_ratio(traffic_1, traffic_2):
    """Eq. (1): for a memory-bound operation P_1 / P_2 = T_2 / T_1."""
    return Fraction(traffic_2) / Fraction(traffic_1)


def matrix_traffic(nrows: int, nnz: int, oindex_bytes: int, iindex_bytes: int, scalar_bytes: int):
    """Eq. (3): bytes of a (DA-)CSR matrix: (nrows + 1) * |oindex_t| +
    nnz * (|iindex_t| + |scalar_t|)."""
    return (nrows + 1) * oindex_bytes + nnz * (iindex_bytes + scalar_bytes)


def spmv_work(nnz: int, nrows: int) -> int:
    """Section 4: W = 2 nnz + 2 nrows floating-point operations."""
    return 2 * nnz + 2 * nrows


def spmv_traffic(nrows: int, ncols: int, nnz: int, oindex_bytes: int, iindex_bytes: int,
                 scalar_bytes: int, vector_bytes: int | None = None, beta_nonzero: bool = False) -> int:
    """Section 4: SpMV traffic = the three arrays of the matrix (Eq. (3)) plus
    x and y.  Reading: x is counted once (ncols entries), y once as written
    (nrows entries) and once more as read when beta != 0.  ``vector_bytes``
    defaults to the matrix scalar size."""
    if vector_bytes is None:
        vector_bytes = scalar_bytes
    t = matrix_traffic(nrows, nnz, oindex_bytes, iindex_bytes, scalar_bytes)
    t += ncols * vector_bytes + nrows * vector_bytes
    if beta_nonzero:
        t += nrows * vector_bytes
    return t


def relative_performance(t_baseline, t_candidate):
    """Section 4: P_candidate / P_baseline = t_baseline / t_candidate (equal work)."""
    return Fraction(t_baseline) / Fraction(t_candidate)


def relative_throughput(traffic_candidate, traffic_baseline, t_baseline, t_candidate):
    """Section 4: (T_candidate / T_baseline) * (t_baseline / t_candidate)."""
    return (Fraction(traffic_candidate) / Fraction(traffic_baseline)) * (
        Fraction(t_baseline) / Fraction(t_candidate))


def approx_traffic_ratio(index_from: str, scalar_from: str, index_to: str, scalar_to: str):
    """Fig. 3: approximate matrix traffic ratio T_to / T_from when the row
    pointer traffic is ignored (|oindex_t| = 0), i.e. bytes per entry
    (|iindex_t| + |scalar_t|) of the target over those of the source."""
    b_from = INDEX_BYTES[index_from] + SCALAR_BYTES[scalar_from]
    b_to = INDEX_BYTES[index_to] + SCALAR_BYTES[scalar_to]
    return Fraction(b_to, b_from)


def predicted_speedup(index_from: str, scalar_from: str, index_to: str, scalar_to: str):
    """Eq. (1) applied to the Fig. 3 ratio: predicted speedup T_from / T_to."""
    return 1 / approx_traffic_ratio(index_from, scalar_from, index_to, scalar_to)


def bytes_per_entry(nrows: int, nnz: int, oindex_bytes: int, iindex_bytes: int):
    """Bookkeeping bytes per stored entry: ((nrows+1)|oindex| + nnz |iindex|) / nnz."""
    return Fraction((nrows + 1) * oindex_bytes + nnz * iindex_bytes, nnz)
