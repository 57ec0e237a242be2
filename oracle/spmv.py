"""y <- alpha A x + beta y for CSR and DA-CSR storage (Section 4, Listing 2).
Test infrastructure only (see ``oracle/__init__.py``).

Listing 2 walks the rows in order.  Each row's sum starts at zero and takes
value * x[col] for the row's entries in stored order; the row's output is
then alpha times that sum, plus beta times the old y entry.  DA-CSR reads x through a view
shifted by the row, so an entry with stored index ``off`` multiplies
x[row + off]; CSR reads x[col] directly.  Both variants compute the same
numbers in the same order.

Readings of points the paper leaves open:

* Products and sums are separately rounded (no fused multiply-add); NumPy's
  element-wise operations do exactly that.  The paper compiles with
  ``-mfma``, so its own rounding is not pinned down.
* beta == 0 follows the BLAS convention: y is output only and is not read
  (NaN or Inf in y is ignored); otherwise the update is alpha*acc + beta*y.
* Non-square matrices: x has ncols entries and is indexed only at row+off /
  col (Remark 3); y has nrows entries.

Besides the Listing 2 order the module gives the exact result (rational
arithmetic, rounded once) and a componentwise error bound that any summation
order satisfies, used as the GPU tolerance:

    |y_gpu - y_exact| <= 4 * nnz_row * 2^-53 * sum_j |a_rj x_j|        (alpha=1, beta=0)
    |y_gpu - y_exact| <= 4 * (nnz_row + 2) * u * (|alpha| sum_j |a_rj x_j| + |beta| |y_r|)

with u = 2^-53 for FP64 accumulation and 2^-24 for FP32.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from .dacsr import entry_rows

U64 = 2.0 ** -53
U32 = 2.0 ** -24
UBF16 = 2.0 ** -8


def _columns(nrows: int, rowptr, idx, diagonal_addressed: bool) -> np.ndarray:
    idx = np.asarray(idx, dtype=np.int64)
    if diagonal_addressed:
        return entry_rows(nrows, rowptr) + idx
    return idx


def spmv_rows(nrows: int, rowptr, idx, val, x, y=None, alpha=1.0, beta=0.0,
              diagonal_addressed: bool = True, dtype=np.float64) -> np.ndarray:
    """Listing 2, one row at a time in pure Python (small inputs).

    ``dtype`` is the accumulation / vector type: float64, or float32 for the
    reduced-precision variant (then every product and sum is rounded to
    FP32)."""
    t = np.dtype(dtype).type
    rowptr = [int(v) for v in rowptr]
    out = np.zeros(nrows, dtype=dtype)
    a = t(alpha)
    b = t(beta)
    for row in range(nrows):
        acc = t(0.0)
        for i in range(rowptr[row], rowptr[row + 1]):
            c = row + int(idx[i]) if diagonal_addressed else int(idx[i])
            acc = t(acc + t(t(val[i]) * t(x[c])))
        if beta == 0:
            out[row] = t(a * acc)
        else:
            out[row] = t(t(a * acc) + t(b * t(y[row])))
    return out


def spmv(nrows: int, rowptr, idx, val, x, y=None, alpha=1.0, beta=0.0,
         diagonal_addressed: bool = True, dtype=np.float64) -> np.ndarray:
    """Listing 2 evaluated for all rows at once: the j-th step adds the j-th
    product of every row that has at least j+1 entries, so each row sees the
    same operations in the same order as ``spmv_rows``."""
    t = np.dtype(dtype).type
    rowptr = np.asarray(rowptr, dtype=np.int64)
    lens = np.diff(rowptr)
    val = np.asarray(val).astype(dtype)
    x = np.asarray(x).astype(dtype)
    cols = _columns(nrows, rowptr, idx, diagonal_addressed)
    acc = np.zeros(nrows, dtype=dtype)
    maxlen = int(lens.max()) if nrows > 0 else 0
    for j in range(maxlen):
        rows_j = np.nonzero(lens > j)[0]
        i = rowptr[rows_j] + j
        acc[rows_j] = acc[rows_j] + val[i] * x[cols[i]]
    if beta == 0:
        return (t(alpha) * acc).astype(dtype)
    return (t(alpha) * acc + t(beta) * np.asarray(y).astype(dtype)).astype(dtype)


def spmv_exact(nrows: int, rowptr, idx, val, x, y=None, alpha=1.0, beta=0.0,
               diagonal_addressed: bool = True, rows=None) -> np.ndarray:
    """alpha A x + beta y in exact rational arithmetic, rounded once to FP64
    (``rows`` restricts the evaluation to a subset)."""
    if rows is None:
        rows = range(nrows)
    a = Fraction(float(alpha))
    b = Fraction(float(beta))
    out = np.zeros(len(rows))
    for k, row in enumerate(rows):
        s = Fraction(0)
        for i in range(int(rowptr[row]), int(rowptr[row + 1])):
            c = row + int(idx[i]) if diagonal_addressed else int(idx[i])
            s += Fraction(float(val[i])) * Fraction(float(x[c]))
        tot = a * s
        if beta != 0:
            tot += b * Fraction(float(y[row]))
        out[k] = float(tot)
    return out


def abs_row_sums(nrows: int, rowptr, idx, val, x, diagonal_addressed: bool = True) -> np.ndarray:
    """sum_j |a_rj x_j| per row (FP64, only used to size tolerances)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    cols = _columns(nrows, rowptr, idx, diagonal_addressed)
    prod = np.abs(np.asarray(val, dtype=np.float64) * np.asarray(x, dtype=np.float64)[cols])
    out = np.zeros(nrows)
    np.add.at(out, entry_rows(nrows, rowptr), prod)
    return out


def error_bound(nrows: int, rowptr, idx, val, x, y=None, alpha=1.0, beta=0.0,
                diagonal_addressed: bool = True, u: float = U64) -> np.ndarray:
    """Componentwise tolerance against the exact result (module docstring).
    A tiny absolute term covers products in the subnormal range."""
    lens = np.diff(np.asarray(rowptr, dtype=np.int64)).astype(np.float64)
    s = abs_row_sums(nrows, rowptr, idx, val, x, diagonal_addressed)
    tiny = np.finfo(np.float64 if u == U64 else np.float32).tiny
    if alpha == 1.0 and beta == 0.0:
        return 4.0 * lens * u * s + lens * tiny
    yabs = np.abs(np.asarray(y, dtype=np.float64)) if beta != 0 else 0.0
    return 4.0 * (lens + 2.0) * u * (abs(alpha) * s + abs(beta) * yabs) + (lens + 2.0) * tiny


def round_to_bf16(v) -> np.ndarray:
    """Round FP64 values to the nearest bfloat16 (8 significant bits, the FP32
    exponent range), ties to even, in one rounding step; returned as FP64.

    The representable neighbours of |v| in [2^e, 2^(e+1)) are spaced 2^(e-7)
    apart (exponent clamped at -126 for the subnormal range); dividing by the
    spacing, rounding to the nearest integer with ties to even and scaling
    back is exact in FP64.  Results beyond the largest finite bfloat16 become
    infinities."""
    v = np.asarray(v, dtype=np.float64)
    out = v.copy()
    fin = np.isfinite(v) & (v != 0)
    m, ex = np.frexp(v[fin])             # v = m * 2^ex, 0.5 <= |m| < 1
    e = np.maximum(ex - 1, -126)         # floor(log2 |v|), clamped
    spacing = np.ldexp(1.0, e - 7)
    r = np.rint(v[fin] / spacing) * spacing
    bf16_max = np.ldexp(2.0 - 2.0 ** -7, 127)
    r = np.where(np.abs(r) > bf16_max, np.copysign(np.inf, r), r)
    out[fin] = r
    return out


UF8 = 2.0 ** -4        # unit roundoff of FP8 E4M3 (3 stored significand bits)
F8_TINY_ABS = 2.0 ** -10  # largest rounding error of an E4M3 subnormal


def round_to_e4m3(v) -> np.ndarray:
    """Round FP64 values to the nearest FP8 E4M3 value, ties to even, in one
    rounding step; returned as FP64.

    E4M3 (the 'fn' variant: no infinities) has a sign bit, 4 exponent bits
    with bias 7 and 3 significand bits: normal values (1 + m/8) 2^(e-7) for
    exponent fields e = 1..15, except that e = 15 with m = 7 encodes NaN, so
    the largest finite value is 1.75 * 2^8 = 448; subnormals m/8 * 2^-6
    (spacing 2^-9).  The neighbours of |v| in [2^e, 2^(e+1)) are 2^(e-3)
    apart (e clamped at -6 for the subnormal range); v / spacing rounded to
    the nearest integer with ties to even and scaled back is exact in FP64.
    A result beyond 448 (|v| > 464, the midpoint to the next binade's first
    step), an infinity or a NaN becomes NaN, the format having no infinity."""
    v = np.asarray(v, dtype=np.float64)
    out = np.full(v.shape, np.nan)
    fin = np.isfinite(v)
    out[fin & (v == 0)] = v[fin & (v == 0)]
    nz = fin & (v != 0)
    m, ex = np.frexp(v[nz])              # v = m * 2^ex, 0.5 <= |m| < 1
    e = np.maximum(ex - 1, -6)           # floor(log2 |v|), clamped
    spacing = np.ldexp(1.0, e - 3)
    r = np.rint(v[nz] / spacing) * spacing
    out[nz] = np.where(np.abs(r) > 448.0, np.nan, r)
    return out


def quantize(val, dtype: str) -> np.ndarray:
    """FP64 values stored in a reduced type (round to nearest, ties to even),
    returned in FP64.  dtype: 'f64', 'f32', 'bf16' or 'f8e4m3'."""
    val = np.asarray(val, dtype=np.float64)
    if dtype == "f64":
        return val.copy()
    if dtype == "f32":
        return val.astype(np.float32).astype(np.float64)
    if dtype == "bf16":
        return round_to_bf16(val)
    if dtype == "f8e4m3":
        return round_to_e4m3(val)
    raise ValueError(dtype)


def spmv_lowp(nrows: int, rowptr, idx, val_lowp, x32, y32=None, alpha=1.0, beta=0.0,
              diagonal_addressed: bool = True) -> np.ndarray:
    """Reduced-precision SpMV: values already rounded to FP32 or BF16 (both
    exact in FP32), x and y in FP32, FP32 accumulation in Listing 2 order."""
    return spmv(nrows, rowptr, idx, np.asarray(val_lowp, dtype=np.float32),
                np.asarray(x32, dtype=np.float32), y32, alpha, beta, diagonal_addressed,
                dtype=np.float32)


def spmm(nrows: int, rowptr, idx, val, X, diagonal_addressed: bool = True,
         dtype=np.float64) -> np.ndarray:
    """Multi-right-hand-side product Y = A X, X row-major [ncols, k]: Listing 2
    applied to every column of X."""
    X = np.asarray(X)
    k = X.shape[1]
    Y = np.zeros((nrows, k), dtype=dtype)
    for j in range(k):
        Y[:, j] = spmv(nrows, rowptr, idx, val, X[:, j], diagonal_addressed=diagonal_addressed,
                       dtype=dtype)
    return Y
