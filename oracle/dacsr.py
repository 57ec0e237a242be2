"""Matrix bandwidth and the CSR -> DA-CSR index translation (Section 2).
Test infrastructure only (see ``oracle/__init__.py``).

CSR stores, for the i-th stored entry, its column c_i; DA-CSR stores c_i - r_i
instead, where r_i is the entry's row (Section 2, Example 1).  Entry order and
values are unchanged.  Explicitly stored zeros count as entries (footnote to
Example 2).

Reading of the 16-bit fit rule: the paper states that a bandwidth below 2^15
admits 16-bit indices (Example 2, Section 3).  The oracle declares a matrix to
fit iff every translated index lies in [-32768, 32767], the range a signed
16-bit integer holds; this differs from "w < 2^15" only when the most negative
offset is exactly -32768.  The same rule with 8 bits ([-128, 127]) gives
DA-CSR-8, the int8 index width of the traffic lattice (Section 2, Fig. 3).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

INT16_MIN = -(1 << 15)
INT16_MAX = (1 << 15) - 1
INT8_MIN = -(1 << 7)
INT8_MAX = (1 << 7) - 1


def entry_rows(nrows: int, rowptr) -> np.ndarray:
    """r_i for every stored entry i: row r owns entries rowptr[r] .. rowptr[r+1]-1."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    return np.repeat(np.arange(nrows, dtype=np.int64), np.diff(rowptr))


def bandwidth(nrows: int, rowptr, col) -> int:
    """Eq. (2): w = max |c - r| over the stored entries (0 for an empty matrix)."""
    col = np.asarray(col, dtype=np.int64)
    if col.size == 0:
        return 0
    return int(np.max(np.abs(col - entry_rows(nrows, rowptr))))


def translate(nrows: int, rowptr, col) -> np.ndarray:
    """Section 2: DA-CSR column ids c_i - r_i, as int64 (not yet narrowed)."""
    col = np.asarray(col, dtype=np.int64)
    return col - entry_rows(nrows, rowptr)


def untranslate(nrows: int, rowptr, off) -> np.ndarray:
    """Inverse of ``translate``: c_i = r_i + off_i."""
    return np.asarray(off, dtype=np.int64) + entry_rows(nrows, rowptr)


@dataclass
class FitInfo:
    min_off: int     # smallest c - r (0 for an empty matrix)
    max_off: int     # largest c - r (0 for an empty matrix)
    w: int           # Eq. (2) bandwidth, max |c - r|
    n_fit: int       # entries whose c - r lies in the offset type's range
    n_bad: int       # entries whose column lies outside [0, ncols)
    fits: bool       # every entry fits and every column is in range


def fit_check(nrows: int, ncols: int, rowptr, col, bits: int = 16) -> FitInfo:
    """Fit information for offsets of a signed ``bits``-bit type (16 or 8)."""
    tmin, tmax = (INT16_MIN, INT16_MAX) if bits == 16 else (INT8_MIN, INT8_MAX)
    off = translate(nrows, rowptr, col)
    c = np.asarray(col, dtype=np.int64)
    n_bad = int(np.count_nonzero((c < 0) | (c >= ncols)))
    if off.size == 0:
        return FitInfo(0, 0, 0, 0, n_bad, n_bad == 0)
    lo, hi = int(off.min()), int(off.max())
    n_fit = int(np.count_nonzero((off >= tmin) & (off <= tmax)))
    return FitInfo(lo, hi, int(max(-lo, hi)), n_fit, n_bad,
                   bool(n_bad == 0 and lo >= tmin and hi <= tmax))


def to_dacsr16(nrows: int, ncols: int, rowptr, col):
    """CSR -> DA-CSR-16.  Returns (off int16 array or None, FitInfo); the
    offsets are returned only when the matrix fits."""
    info = fit_check(nrows, ncols, rowptr, col)
    if not info.fits:
        return None, info
    return translate(nrows, rowptr, col).astype(np.int16), info


def to_dacsr8(nrows: int, ncols: int, rowptr, col):
    """CSR -> DA-CSR-8 (int8 offsets).  Returns (off int8 array or None,
    FitInfo for 8 bits)."""
    info = fit_check(nrows, ncols, rowptr, col, bits=8)
    if not info.fits:
        return None, info
    return translate(nrows, rowptr, col).astype(np.int8), info
