"""Pins of the BSR / DA-BSR oracle: expansion to scalar CSR against a dense
matrix written entry by entry, DA translation of the block pattern, and a
2 x 2 example worked by hand."""
import numpy as np
import pytest

import workloads as W
from oracle import bsr as B
from oracle import dacsr as D
from oracle import spmv as S


def test_hand_example():
    # blocks: (0,0) [[1,2],[3,4]], (0,1) [[5,6],[7,8]], (1,1) [[9,10],[11,12]]
    browptr = np.array([0, 2, 3])
    bcol = np.array([0, 1, 1])
    bval = np.arange(1, 13, dtype=float).reshape(3, 2, 2)
    rp, col, val = B.expand(2, 2, browptr, bcol, bval)
    assert rp.tolist() == [0, 4, 8, 10, 12]
    assert col.tolist() == [0, 1, 2, 3, 0, 1, 2, 3, 2, 3, 2, 3]
    assert val.tolist() == [1, 2, 5, 6, 3, 4, 7, 8, 9, 10, 11, 12]
    x = np.array([1.0, 10.0, 100.0, 1000.0])
    y = S.spmv(4, rp, col, val, x, diagonal_addressed=False)
    assert y.tolist() == [1 + 20 + 500 + 6000, 3 + 40 + 700 + 8000, 900 + 10000, 1100 + 12000]
    off = D.translate(2, browptr, bcol)
    assert off.tolist() == [0, 1, 0]
    rp2, col2, _ = B.expand(2, 2, browptr, off, bval, diagonal_addressed=True)
    assert np.array_equal(col2, col) and np.array_equal(rp2, rp)


@pytest.mark.parametrize("b", [2, 3, 4])
def test_expand_matches_dense(b):
    m = 4
    nbr, browptr, bcol, bval = W.block_stencil3d(m, b, np.random.default_rng(b))
    rp, col, val = B.expand(nbr, b, browptr, bcol, bval)
    A = B.dense(nbr, nbr, b, browptr, bcol, bval)
    x = np.random.default_rng(7).uniform(-1, 1, nbr * b)
    y = S.spmv(nbr * b, rp, col, val, x, diagonal_addressed=False)
    assert np.allclose(y, A @ x, rtol=1e-13, atol=1e-12)
    # DA-BSR: offsets of the block pattern expand to the same scalar matrix
    off = D.translate(nbr, browptr, bcol)
    rp2, col2, val2 = B.expand(nbr, b, browptr, off, bval, diagonal_addressed=True)
    assert np.array_equal(rp2, rp) and np.array_equal(col2, col) and np.array_equal(val2, val)
    # the block bandwidth is the grid's m^2, the scalar one about b times larger
    assert D.bandwidth(nbr, browptr, bcol) == m * m
