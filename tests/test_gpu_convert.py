"""GPU parity of the CSR -> DA-CSR-16 translation and fit check (Section 2,
Example 1) against the oracle: bit-exact offsets and fit information."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import dacsr as OD
from oracle import spmv as OS

pytestmark = pytest.mark.gpu


def _to(dev, *arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrs]


def _check(D, dev, n_rows, n_cols, rp, col):
    t_rp, t_col = _to(dev, rp, col)
    off, info = D.damn_csr_to_dacsr(t_rp, t_col, n_cols)
    ref = OD.fit_check(n_rows, n_cols, rp, col)
    assert (info.min_off, info.max_off, info.w, info.n_fit, info.n_bad, info.fits) == \
        (ref.min_off, ref.max_off, ref.w, ref.n_fit, ref.n_bad, ref.fits)
    if ref.fits:
        assert np.array_equal(off.cpu().numpy(), OD.translate(n_rows, rp, col).astype(np.int16))
    return info


def test_example1(D, cuda_dev, golden):
    g = golden("example1_dacsr.txt")
    rp = np.array(g["rowptr"], dtype=np.int32)
    col = np.array(g["colids_csr"], dtype=np.int32)
    info = _check(D, cuda_dev, 4, 4, rp, col)
    t_rp, t_col = _to(cuda_dev, rp, col)
    off, _ = D.damn_csr_to_dacsr(t_rp, t_col, 4)
    assert off.cpu().tolist() == [int(v) for v in g["colids_dacsr"]]
    assert info.w == 1


@pytest.mark.parametrize("n,h,seed", [(1, 1, 0), (511, 3, 1), (513, 40, 2), (5000, 100, 3),
                                      (40000, 1000, 4), (100003, 30000, 5)])
def test_random_banded(D, cuda_dev, n, h, seed):
    rp, col, _ = W.random_banded(n, h, np.random.default_rng(seed))
    _check(D, cuda_dev, n, n, rp, col)


@pytest.mark.parametrize("extreme", [32767, -32768, 32768, -32769, 100000])
def test_fit_boundary(D, cuda_dev, extreme):
    n = 140000
    r = 70000
    rows = np.append(np.arange(n), r)
    cols = np.append(np.arange(n), r + extreme)
    rp, col, _ = W.from_coo(n, rows, cols)
    info = _check(D, cuda_dev, n, n, rp, col)
    assert info.fits == (-32768 <= extreme <= 32767)


def test_empty_rows_nonsquare_and_bad_columns(D, cuda_dev):
    rp = np.zeros(10, dtype=np.int32)
    _check(D, cuda_dev, 9, 5, rp, np.zeros(0, dtype=np.int32))
    rp, col, _ = W.from_coo(700, [0, 3, 5, 5, 699], [0, 1, 0, 2, 2])
    _check(D, cuda_dev, 700, 3, rp, col)
    info = _check(D, cuda_dev, 700, 2, rp, col)      # column 2 out of range
    assert info.n_bad == 2 and not info.fits


def test_bad_column_near_int_min(D, cuda_dev):
    """c - r is formed in 64 bits: a column of -2^31 in row 5 gives c - r =
    -2^31 - 5, which the int32 min_off reports saturated at -2^31; the
    counts and the fit decision are exact."""
    n = 700
    rows = np.append(np.arange(n), [5, 600])
    cols = np.append(np.arange(n), [-2 ** 31, 2 ** 31 - 1]).astype(np.int64)
    rp, col, _ = W.from_coo(n, rows, cols)
    col = col.astype(np.int32)
    t_rp, t_col = _to(cuda_dev, rp, col)
    for convert, bits in ((D.damn_csr_to_dacsr, 16), (D.damn_csr_to_dacsr_noalloc, 16)):
        if convert is D.damn_csr_to_dacsr_noalloc:
            out = torch.empty(len(col), dtype=torch.int16, device=cuda_dev)
            _, info = convert(t_rp, t_col, n, out)
        else:
            _, info = convert(t_rp, t_col, n)
        ref = OD.fit_check(n, n, rp, col, bits=bits)
        assert ref.min_off == -2 ** 31 - 5 and ref.max_off == 2 ** 31 - 1 - 600
        sat = lambda v: max(-2 ** 31, min(2 ** 31 - 1, v))
        assert (info.min_off, info.max_off, info.n_fit, info.n_bad, info.fits) == \
            (sat(ref.min_off), sat(ref.max_off), ref.n_fit, ref.n_bad, False)
        assert info.w == 2 ** 31


def test_laplace3d_full_size_and_scrambled(D, cuda_dev):
    m = 128
    rp, col, _ = W.laplace3d_7pt(m)
    info = _check(D, cuda_dev, m ** 3, m ** 3, rp, col)
    assert info.fits and info.w == m * m
    rp2, col2, _ = W.laplace3d_7pt(m, scrambled=True, rng=W.rng_for(2, 1))
    info2 = _check(D, cuda_dev, m ** 3, m ** 3, rp2, col2)
    assert not info2.fits
    rate = info2.n_fit / len(col2)
    assert 0.15 < rate < 0.20     # diagonal (1/7) plus ~3% of the off-diagonals


def test_validate_csr(D, cuda_dev):
    rp, col, _ = W.random_banded(3000, 50, np.random.default_rng(9))
    t_rp, t_col = _to(cuda_dev, rp, col)
    assert D.damn_validate_csr(t_rp, t_col, 3000) == (0, 0)
    bad_rp = rp.copy()
    bad_rp[10] = bad_rp[11] + 1
    bad_col = col.copy()
    bad_col[[5, 7]] = [-1, 3000]
    t_rp, t_col = _to(cuda_dev, bad_rp, bad_col)
    br, bc = D.damn_validate_csr(t_rp, t_col, 3000)
    assert br >= 1 and bc == 2


def test_validate_dacsr(D, cuda_dev):
    """r + off inside [0, ncols) for every entry, for int16 and int8 offsets;
    out-of-range addresses and broken row pointers are counted, not read."""
    n = 3000
    rp, col, _ = W.random_banded(n, 50, np.random.default_rng(19))
    off = OD.translate(n, rp, col)
    t_rp = _to(cuda_dev, rp)[0]
    assert D.damn_validate_dacsr(t_rp, _to(cuda_dev, off.astype(np.int16))[0], n) == (0, 0)
    rp8, col8, _ = W.random_banded(n, 100, np.random.default_rng(20))
    off8 = OD.translate(n, rp8, col8)
    assert np.abs(off8).max() <= 127
    assert D.damn_validate_dacsr(_to(cuda_dev, rp8)[0], _to(cuda_dev, off8.astype(np.int8))[0],
                                 n) == (0, 0)
    bad = off.copy()
    bad[0] = -5                 # row 0: column -5
    bad[-1] = 10               # last row: column n + 9
    bad[len(bad) // 2] = 32767  # a middle row: far past ncols
    assert D.damn_validate_dacsr(t_rp, _to(cuda_dev, bad.astype(np.int16))[0], n) == (0, 3)
    # a narrower matrix: every entry with r + off >= ncols counts
    nc = 2000
    want = int(np.count_nonzero(OD.entry_rows(n, rp) + off >= nc))
    assert D.damn_validate_dacsr(t_rp, _to(cuda_dev, off.astype(np.int16))[0], nc)[1] == want
    # broken row pointers: counted; the entry range stays inside off
    brp = rp.copy()
    brp[100] = brp[101] + 7
    brp[-1] = brp[-1] + 1000
    br, _ = D.damn_validate_dacsr(_to(cuda_dev, brp)[0], _to(cuda_dev, off.astype(np.int16))[0], n)
    assert br >= 2


def test_cast_values(D, cuda_dev):
    rng = np.random.default_rng(4)
    v = np.concatenate([rng.standard_normal(100000) * 10.0 ** rng.integers(-40, 40, 100000),
                        [1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -40, 2.0 ** -133,
                         2.0 ** -135, 3.4e38, -3.4e38, 0.0, -0.0, 26.5, -1.0]])
    t = torch.from_numpy(v).to(cuda_dev)
    f32 = D.damn_cast_values(t, torch.float32).double().cpu().numpy()
    assert np.array_equal(f32, OS.quantize(v, "f32"))
    bf = D.damn_cast_values(t, torch.bfloat16).double().cpu().numpy()
    assert np.array_equal(bf, OS.quantize(v, "bf16"))
    # FP8 E4M3 (one rounding step from FP64; beyond 464, inf and NaN -> NaN)
    v8 = np.concatenate([v, rng.uniform(-500, 500, 20000), rng.uniform(-2 ** -5, 2 ** -5, 20000),
                         [1 + 2 ** -4 + 2 ** -30, 464.0, 464.01, 448.0, 2.0 ** -10,
                          3 * 2.0 ** -11, np.inf, -np.inf, np.nan, 1e-310]])
    t8 = torch.from_numpy(v8).to(cuda_dev)
    f8 = D.damn_cast_values(t8, torch.float8_e4m3fn)
    assert np.array_equal(f8.double().cpu().numpy(), OS.quantize(v8, "f8e4m3"), equal_nan=True)
    # the NaN encoding is the format's (S.1111.111), and signed zeros keep their sign
    bits = f8.view(torch.uint8).cpu().numpy()
    assert set(bits[np.isnan(OS.quantize(v8, "f8e4m3"))]) <= {0x7F, 0xFF}
    z = D.damn_cast_values(torch.tensor([-0.0, 0.0, -1e-300], dtype=torch.float64, device=cuda_dev),
                           torch.float8_e4m3fn).view(torch.uint8).cpu().tolist()
    assert z == [0x80, 0x00, 0x80]
    # FP32 -> E4M3 equals torch's own conversion of FP32 values
    v32 = v8[np.isfinite(v8)].astype(np.float32)
    g32 = D.damn_cast_values(torch.from_numpy(v32).to(cuda_dev), torch.float8_e4m3fn)
    ref32 = torch.from_numpy(v32).to(torch.float8_e4m3fn)
    assert np.array_equal(g32.double().cpu().numpy(), ref32.double().numpy(), equal_nan=True)
