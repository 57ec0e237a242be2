"""The seeded generators produce the shapes the workloads state."""
import numpy as np

import workloads as W
from oracle import dacsr as D
from oracle import rcm as R


def _check_csr(n, rp, c, ncols=None):
    ncols = n if ncols is None else ncols
    assert rp.dtype == np.int32 and c.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == len(c) and np.all(np.diff(rp) >= 0)
    assert c.min() >= 0 and c.max() < ncols
    for r in range(0, n, max(1, n // 50)):
        seg = c[rp[r]:rp[r + 1]]
        assert np.all(np.diff(seg) > 0)


def test_laplace2d():
    rp, c, v = W.laplace2d_5pt(64)
    n = 4096
    assert len(c) == 20224
    _check_csr(n, rp, c)
    assert D.bandwidth(n, rp, c) == 64
    assert set(np.unique(v)) == {4.0, -1.0}


def test_laplace3d_natural_and_scrambled():
    m = 10
    n = m ** 3
    rp, c, v = W.laplace3d_7pt(m)
    assert len(c) == 7 * m ** 3 - 6 * m ** 2
    _check_csr(n, rp, c)
    rng = W.rng_for(2, 1)
    rp2, c2, v2 = W.laplace3d_7pt(m, scrambled=True, rng=rng)
    labels = W.rng_for(2, 1).permutation(n)
    # scrambled = P A P^T with new index labels[v] for grid vertex v
    perm = np.argsort(labels)
    rp3, c3, v3 = R.permute_symmetric(n, rp, c, v, perm)
    assert np.array_equal(rp2, rp3) and np.array_equal(c2, c3) and np.array_equal(v2, v3)


def test_stencil27_counts():
    m = 7
    rp, c, v = W.stencil27(m)
    assert len(c) == (3 * m - 2) ** 3
    _check_csr(m ** 3, rp, c)
    assert (3 * 160 - 2) ** 3 == 109215352
    assert D.bandwidth(m ** 3, rp, c) == m * m + m + 1


def test_random_banded_shape():
    rng = W.rng_for(3, 0)
    n, h = 5000, 100
    rp, c, v = W.random_banded(n, h, rng)
    _check_csr(n, rp, c)
    assert D.bandwidth(n, rp, c) <= h
    r = D.entry_rows(n, rp)
    # diagonal present in every row
    assert np.count_nonzero(c == r) == n
    lens = np.diff(rp)
    assert 1 <= lens.min() and lens.max() <= 200
    assert 10 <= np.median(lens) <= 13
    rp2, c2, v2 = W.random_banded(n, h, W.rng_for(3, 0))
    assert np.array_equal(c, c2) and np.array_equal(v, v2)


def test_batch_banded():
    mats = W.batch_banded(6)
    for n, rp, c, v in mats:
        assert 1000 <= n <= 200000
        _check_csr(n, rp, c)
        assert D.bandwidth(n, rp, c) <= 4096
        lens = np.diff(rp)
        assert lens.min() >= 1 and lens.max() <= 40


def test_perturb_symmetric_keeps_symmetry_and_dominance():
    m = 10
    rp, col, val = W.stencil27(m)
    n = m ** 3
    pv = W.perturb_symmetric(n, rp, col, val, sigma=0.01)
    import scipy.sparse as sp
    A = sp.csr_matrix((pv, col, rp), shape=(n, n))
    assert abs(A - A.T).max() == 0.0
    d = A.diagonal()
    assert np.array_equal(d, np.full(n, 26.5))
    off = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(d)
    assert np.all(off < d)                          # strictly diagonally dominant: SPD
    delta = (pv - val)[(pv - val) != 0]
    assert 0.008 < delta.std() < 0.012 and abs(delta.mean()) < 0.002


def test_full_size_workloads_match_their_documented_sizes():
    """The seeded generators give, at full size, the entry counts the
    benchmark's byte model and the design notes quote: the 512-matrix batch
    (12,182,394 rows, 271,862,000 entries, 2.96 GB at FP64 and k = 1) and the
    random banded matrix n = 1e6, h = 1000 (13,551,395 entries)."""
    mats = W.batch_banded(512)
    assert sum(m[0] for m in mats) == 12_182_394
    assert sum(len(m[2]) for m in mats) == 271_862_000
    nbytes = sum((m[0] + 1) * 4 + len(m[2]) * (2 + 8) + 2 * m[0] * 8 for m in mats)
    assert nbytes == 2_962_269_928
    rp, c, _ = W.random_banded(1_000_000, 1000, W.rng_for(3, 0))
    assert len(c) == 13_551_395
    assert 13.0 < len(c) / 1e6 < 14.0
