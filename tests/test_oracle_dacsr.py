"""Pins of the CSR -> DA-CSR translation and the bandwidth (Section 2,
Eq. (2), Example 1)."""
import numpy as np
import pytest

import workloads as W
from oracle import dacsr as D


def test_example1(golden):
    g = golden("example1_dacsr.txt")
    rowptr = np.array(g["rowptr"], dtype=np.int32)
    col = np.array(g["colids_csr"], dtype=np.int32)
    n = int(g["nrows"][0])
    off, info = D.to_dacsr16(n, int(g["ncols"][0]), rowptr, col)
    assert off.tolist() == [int(v) for v in g["colids_dacsr"]]
    assert info.w == int(g["w"][0]) and info.fits
    assert len(col) == int(g["nnz"][0])
    # the generator's copy of Fig. 1 is the same pattern
    rp, c, _ = W.example1_pattern()
    assert rp.tolist() == rowptr.tolist() and c.tolist() == col.tolist()
    # Example 1: the stored indices span [0, ncols-1] in CSR and [-w, w] in DA-CSR
    assert (col.min(), col.max()) == (0, n - 1)
    assert (off.min(), off.max()) == (-info.w, info.w)


def _dense_bandwidth(n_rows, n_cols, rowptr, col):
    """Bandwidth by brute force over a dense 0/1 pattern matrix."""
    P = np.zeros((n_rows, n_cols), dtype=bool)
    for r in range(n_rows):
        P[r, col[rowptr[r]:rowptr[r + 1]]] = True
    rr, cc = np.nonzero(P)
    return int(np.max(np.abs(cc - rr))) if len(rr) else 0


@pytest.mark.parametrize("seed", range(5))
def test_bandwidth_brute_force(seed):
    rng = np.random.default_rng(seed)
    nr, nc = rng.integers(1, 40, size=2)
    nnz = rng.integers(0, nr * nc)
    rows = rng.integers(0, nr, size=nnz)
    cols = rng.integers(0, nc, size=nnz)
    rp, c, _ = W.from_coo(nr, rows, cols)
    assert D.bandwidth(nr, rp, c) == _dense_bandwidth(nr, nc, rp, c)
    off = D.translate(nr, rp, c)
    assert np.array_equal(D.untranslate(nr, rp, off), c)
    # entry-by-entry definition: off_i = c_i - r_i
    for r in range(nr):
        for i in range(rp[r], rp[r + 1]):
            assert off[i] == c[i] - r


def test_explicit_zeros_count():
    # an explicitly stored zero far from the diagonal still sets w
    rp, c, v = W.from_coo(3, [0, 1, 2, 2], [0, 1, 2, 0], [1.0, 1.0, 1.0, 0.0])
    assert D.bandwidth(3, rp, c) == 2


@pytest.mark.parametrize("extreme,fits", [(32767, True), (-32767, True), (-32768, True),
                                          (32768, False), (-32769, False)])
def test_int16_boundary(extreme, fits):
    n = 70000
    r = 33000
    rows = np.arange(n)
    cols = np.arange(n)
    rows = np.append(rows, r)
    cols = np.append(cols, r + extreme)
    rp, c, _ = W.from_coo(n, rows, cols)
    off, info = D.to_dacsr16(n, n, rp, c)
    assert info.fits == fits
    assert info.w == abs(extreme)
    assert info.n_fit == n + (1 if fits else 0)
    if fits:
        assert int(off.min()) == min(0, extreme) and int(off.max()) == max(0, extreme)


def test_empty_and_nonsquare():
    rp = np.zeros(6, dtype=np.int32)
    info = D.fit_check(5, 3, rp, np.zeros(0, dtype=np.int32))
    assert info.fits and info.w == 0 and info.n_fit == 0
    # tall matrix (Remark 3): nrows > ncols
    rp, c, _ = W.from_coo(6, [0, 3, 5, 5], [0, 1, 0, 2])
    off, info = D.to_dacsr16(6, 3, rp, c)
    assert off.tolist() == [0, -2, -5, -3]
    assert info.fits and info.w == 5
    # a column outside [0, ncols) makes the conversion fail
    info = D.fit_check(6, 2, rp, c)
    assert info.n_bad == 1 and not info.fits


def test_workload_fit_rates():
    # 7-point Laplacian on a small grid: natural order has w = m^2
    m = 12
    rp, c, _ = W.laplace3d_7pt(m)
    assert D.bandwidth(m ** 3, rp, c) == m * m
    assert len(c) == 7 * m ** 3 - 6 * m ** 2


@pytest.mark.parametrize("extreme,fits", [(127, True), (-127, True), (-128, True),
                                          (128, False), (-129, False)])
def test_int8_boundary(extreme, fits):
    """DA-CSR-8: the same rule over [-128, 127]."""
    n = 400
    r = 200
    rows = np.append(np.arange(n), r)
    cols = np.append(np.arange(n), r + extreme)
    rp, c, _ = W.from_coo(n, rows, cols)
    off, info = D.to_dacsr8(n, n, rp, c)
    assert info.fits == fits
    assert info.w == abs(extreme)
    assert info.n_fit == n + (1 if fits else 0)
    if fits:
        assert off.dtype == np.int8
        assert int(off.min()) == min(0, extreme) and int(off.max()) == max(0, extreme)
        assert np.array_equal(D.untranslate(n, rp, off), c)


def test_int8_fit_of_grids():
    # 2-D 5-point Laplacian: w = m, so DA-CSR-8 holds up to m = 127
    for m, fits in ((127, True), (128, False)):
        rp, c, _ = W.laplace2d_5pt(m)
        assert D.fit_check(m * m, m * m, rp, c, bits=8).fits == fits
        assert D.fit_check(m * m, m * m, rp, c, bits=16).fits


@pytest.mark.parametrize("mistake", ["sign", "row_shift", "w_without_abs", "symmetric_fit",
                                     "strict_upper"])
def test_planted_mistakes_are_caught(mistake, monkeypatch, golden):
    """Each plausible slip in the translation or the fit rule fails one of the
    pins above (the mistake is planted in the oracle, on the CPU)."""
    if mistake == "sign":
        monkeypatch.setattr(D, "translate", lambda n, rp, c: D.entry_rows(n, rp) - np.asarray(c))
    elif mistake == "row_shift":
        real = D.entry_rows
        monkeypatch.setattr(D, "entry_rows", lambda n, rp: np.minimum(real(n, rp) + 1, n - 1))
    elif mistake == "w_without_abs":
        monkeypatch.setattr(D, "bandwidth", lambda n, rp, c: int(np.max(D.translate(n, rp, c)))
                            if len(c) else 0)
    elif mistake == "symmetric_fit":
        monkeypatch.setattr(D, "INT16_MIN", -32767)
    else:
        monkeypatch.setattr(D, "INT16_MAX", 32766)
    pins = [lambda: test_example1(golden),
            lambda: [test_bandwidth_brute_force(s) for s in range(5)],
            test_explicit_zeros_count,
            lambda: [test_int16_boundary(e, f) for e, f in
                     ((32767, True), (-32767, True), (-32768, True), (32768, False),
                      (-32769, False))]]
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, mistake
