"""The allocation-free conversion entry point, damn_csr_to_dacsr_noalloc.

It exists for callers that cannot allocate device memory (their framework
owns every device allocation, or cudaMalloc's device-wide synchronisation is
not acceptable on their path); its scratch is a static array inside the
library.  This checks, through the C ABI, that two calls in a row each give
exactly the output of the workspace-based damn_csr_to_dacsr (offsets are
integers, so bit for bit), that stale scratch from the first call does not
leak into the second, and that matrices beyond its row limit are refused.

The file name makes pytest collect it last.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import dacsr as OD

pytestmark = pytest.mark.gpu


def _t(dev, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _compare(D, dev, n_rows, n_cols, rp, col):
    t_rp, t_col = _t(dev, rp), _t(dev, col)
    ref_off, ref = D.damn_csr_to_dacsr(t_rp, t_col, n_cols)
    off = torch.full((len(col),), -7, dtype=torch.int16, device=dev)
    got_off, got = D.damn_csr_to_dacsr_noalloc(t_rp, t_col, n_cols, off)
    torch.cuda.synchronize()
    assert got == ref
    # and against the CPU oracle's fit check and translation
    o = OD.fit_check(n_rows, n_cols, rp, col)
    assert (got.min_off, got.max_off, got.w, got.n_fit, got.n_bad, bool(got.fits)) == \
        (o.min_off, o.max_off, o.w, o.n_fit, o.n_bad, o.fits)
    if ref.fits:
        assert torch.equal(got_off, ref_off)
        assert np.array_equal(got_off.cpu().numpy(),
                              OD.translate(n_rows, rp, col).astype(np.int16))
    return got


def test_two_calls_match_workspace_entry(D, cuda_dev):
    # first call: a large banded matrix that fits int16
    n1 = 600_000
    rp1, col1, _ = W.random_banded(n1, 2000, np.random.default_rng(41))
    info1 = _compare(D, cuda_dev, n1, n1, rp1, col1)
    assert info1.fits and info1.w <= 2000
    # second call right after, smaller and not fitting: the result must not
    # carry anything over from the first call's scratch contents
    n2 = 90_001
    rows = np.append(np.arange(n2), [5, n2 - 1])
    cols = np.append(np.arange(n2), [5 + 40_000, n2 - 1 - 50_000])
    rp2, col2, _ = W.from_coo(n2, rows, cols)
    info2 = _compare(D, cuda_dev, n2, n2, rp2, col2)
    assert not info2.fits and info2.min_off == -50_000 and info2.max_off == 40_000


def test_row_limit_and_empty(D, cuda_dev):
    # empty matrix
    rp = np.zeros(11, dtype=np.int32)
    info = _compare(D, cuda_dev, 10, 10, rp, np.zeros(0, dtype=np.int32))
    assert info.fits and info.w == 0
    # beyond the static scratch: refused before any device work
    n = D.DAMN_NOALLOC_MAX_ROWS + 1
    t_rp = torch.zeros(2, dtype=torch.int32, device=cuda_dev)
    t_col = torch.zeros(1, dtype=torch.int32, device=cuda_dev)
    off = torch.zeros(1, dtype=torch.int16, device=cuda_dev)
    info = D.damn_fit_info()
    import ctypes
    rc = D._lib.damn_csr_to_dacsr_noalloc(n, n, 0, D._ptr(t_rp), D._ptr(t_col), D._ptr(off),
                                          ctypes.byref(info), D._stream())
    assert rc == D.DAMN_ERR_INVALID_ARG
    assert "static scratch" in D.last_error()
    assert D.damn_device_status() == 0
