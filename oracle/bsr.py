"""Block CSR (BSR) and its diagonally-addressed form DA-BSR.
Test infrastructure only (see ``oracle/__init__.py``).

The paper notes that diagonal addressing applies to other sparse formats,
BSR among them (Section 1).  In BSR the matrix is a grid of b x b blocks;
block row R stores, for each of its non-zero blocks k, the block column C_k
and the b*b values (row-major inside the block).  DA-BSR stores C_k - R
instead of C_k, i.e. Section 2's translation applied to the block pattern,
so one 16-bit (or 8-bit) index serves b*b values.

y = A x in BSR is, per scalar row r = R*b + i, the sum over the row's blocks
k (stored order) and the block columns j = 0..b-1 (ascending) of
val[k, i, j] * x[C_k*b + j].  ``expand`` writes exactly that as a scalar CSR
matrix (entries of scalar row r in the order (k, j)), so the CSR oracle's
Listing 2 loop, exact product and error bound apply unchanged.
"""
from __future__ import annotations

import numpy as np

from .dacsr import entry_rows


def expand(nbr: int, b: int, browptr, bidx, bval, diagonal_addressed: bool = False):
    """Scalar CSR (rowptr, col, val) of a BSR / DA-BSR matrix, entries of
    each scalar row in (block, column-in-block) order."""
    browptr = np.asarray(browptr, dtype=np.int64)
    bidx = np.asarray(bidx, dtype=np.int64)
    bval = np.asarray(bval).reshape(-1, b, b)
    brow = entry_rows(nbr, browptr)
    bcol = brow + bidx if diagonal_addressed else bidx
    nblk = len(bcol)
    cnt = np.diff(browptr)                              # blocks per block row
    rowptr = np.zeros(nbr * b + 1, dtype=np.int64)
    np.cumsum(np.repeat(cnt * b, b), out=rowptr[1:])
    # scalar row R*b+i holds, for each block k of block row R, the b entries
    # (k, i, 0..b-1): build them block row by block row
    col = np.empty(nblk * b * b, dtype=np.int64)
    val = np.empty(nblk * b * b, dtype=bval.dtype)
    for R in range(nbr):
        k0, k1 = browptr[R], browptr[R + 1]
        nb = k1 - k0
        for i in range(b):
            s = rowptr[R * b + i]
            cols = (bcol[k0:k1, None] * b + np.arange(b)[None, :]).reshape(-1)
            col[s:s + nb * b] = cols
            val[s:s + nb * b] = bval[k0:k1, i, :].reshape(-1)
    return rowptr.astype(np.int32), col.astype(np.int32), val


def dense(nbr: int, nbc: int, b: int, browptr, bcol, bval) -> np.ndarray:
    """Dense matrix of a BSR matrix, written entry by entry (pins ``expand``)."""
    A = np.zeros((nbr * b, nbc * b))
    bval = np.asarray(bval).reshape(-1, b, b)
    for R in range(nbr):
        for k in range(int(browptr[R]), int(browptr[R + 1])):
            C = int(bcol[k])
            for i in range(b):
                for j in range(b):
                    A[R * b + i, C * b + j] += bval[k, i, j]
    return A
