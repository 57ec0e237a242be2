"""DA-COO (diagonal addressing of COO's column vector) through the C ABI:
COO-32 and DA-COO-16 bitwise equal, bitwise equal to the oracle on dyadic
inputs, within the error bound of the exact product otherwise, empty rows,
rows crossing many chunks, alpha/beta, no entries."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import dacsr as OD
from oracle import spmv as OS

pytestmark = pytest.mark.gpu


def _t(dev, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _matrix(rng, n, long_rows=True):
    lens = rng.integers(0, 25, size=n)
    lens[rng.random(n) < 0.1] = 0                      # empty rows
    if long_rows:
        lens[rng.choice(n, 3, replace=False)] = [300, 1000, 57]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    r = np.repeat(np.arange(n), lens)
    col = np.clip(r + rng.integers(-400, 401, size=len(r)), 0, n - 1).astype(np.int32)
    return rp.astype(np.int32), col


def _run(D, dev, n, rp, col, val, x, alpha=1.0, beta=0.0, y0=None, dt=torch.float64):
    row = OD.entry_rows(n, rp).astype(np.int32)
    off = OD.translate(n, rp, col).astype(np.int16)
    vec = torch.float64 if dt == torch.float64 else torch.float32
    tv = _t(dev, val).to(dt) if dt != torch.bfloat16 else D.damn_cast_values(_t(dev, val), dt)
    ys = []
    for fn, idx in ((D.damn_spmv_coo32, col), (D.damn_spmv_dacoo16, off)):
        y = _t(dev, y0).to(vec) if y0 is not None else torch.full((n,), float("nan"), dtype=vec,
                                                                   device=dev)
        fn(n, _t(dev, row), _t(dev, idx), tv, _t(dev, x).to(vec), y, alpha=alpha, beta=beta)
        ys.append(y)
    torch.cuda.synchronize()
    assert torch.equal(ys[0], ys[1])
    return ys[1].double().cpu().numpy()


def test_dacoo_dyadic_bitwise(D, cuda_dev):
    rng = np.random.default_rng(1)
    n = 3000
    rp, col = _matrix(rng, n)
    val = rng.integers(-4, 5, size=len(col)).astype(np.float64)
    x = W.dyadic_vector(n, rng)
    y = _run(D, cuda_dev, n, rp, col, val, x)
    assert np.array_equal(y, OS.spmv(n, rp, col, val, x, diagonal_addressed=False))


@pytest.mark.parametrize("dt", [torch.float64, torch.float32, torch.bfloat16])
def test_dacoo_random_within_bound(D, cuda_dev, dt):
    rng = np.random.default_rng(2)
    n = 2000
    rp, col = _matrix(rng, n)
    val = rng.standard_normal(len(col))
    x = rng.uniform(-1, 1, n)
    y = _run(D, cuda_dev, n, rp, col, val, x, dt=dt)
    if dt == torch.float64:
        vq, xq, u = val, x, OS.U64
    else:
        vq = OS.quantize(val, "f32" if dt == torch.float32 else "bf16")
        xq, u = x.astype(np.float32).astype(np.float64), OS.U32
    rows = np.arange(0, n, 3)
    ex = OS.spmv_exact(n, rp, col, vq, xq, diagonal_addressed=False, rows=rows)
    bnd = OS.error_bound(n, rp, col, vq, xq, diagonal_addressed=False, u=u)[rows]
    assert np.all(np.abs(y[rows] - ex) <= bnd)
    assert np.all(y[np.diff(rp) == 0] == 0)


def test_dacoo_alpha_beta_and_empty(D, cuda_dev):
    rng = np.random.default_rng(3)
    n = 1500
    rp, col = _matrix(rng, n)
    val = rng.standard_normal(len(col))
    x = rng.uniform(-1, 1, n)
    y0 = rng.uniform(-1, 1, n)
    y = _run(D, cuda_dev, n, rp, col, val, x, alpha=0.75, beta=-1.5, y0=y0)
    ex = OS.spmv_exact(n, rp, col, val, x, y=y0, alpha=0.75, beta=-1.5, diagonal_addressed=False)
    bnd = OS.error_bound(n, rp, col, val, x, y=y0, alpha=0.75, beta=-1.5, diagonal_addressed=False)
    assert np.all(np.abs(y - ex) <= bnd)
    # no entries at all: y = beta y0
    rp0 = np.zeros(n + 1, dtype=np.int32)
    e = np.zeros(0, dtype=np.int32)
    y = _run(D, cuda_dev, n, rp0, e, np.zeros(0), x, beta=2.0, y0=y0)
    assert np.array_equal(y, 2.0 * y0)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_dacoo_tiles_long_rows_gaps_unaligned(D, cuda_dev, dt):
    """Rows longer than a tile of 2048 entries (finished across tiles), a run
    of 3000 empty rows (owned rows beyond one shared-memory window), and
    arrays that are not 16-byte aligned (element loads instead of 16-byte
    loads): dyadic inputs make every summation order exact, so the result
    equals the oracle bitwise on both load paths."""
    rng = np.random.default_rng(5)
    n = 40000
    lens = rng.integers(0, 12, size=n)
    lens[10000:13000] = 0
    lens[20000], lens[20001], lens[30000] = 5000, 2048, 4097
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    rp = rp.astype(np.int32)
    r = np.repeat(np.arange(n), lens)
    col = np.clip(r + rng.integers(-2000, 2001, size=len(r)), 0, n - 1).astype(np.int32)
    val = rng.integers(-4, 5, size=len(col)).astype(np.float64)
    x = W.dyadic_vector(n, rng, bits=8)
    ref = OS.spmv(n, rp, col, val, x, diagonal_addressed=False)
    row = OD.entry_rows(n, rp).astype(np.int32)
    off = OD.translate(n, rp, col).astype(np.int16)
    tx = _t(cuda_dev, x).to(dt)
    outs = []
    for shift in (0, 1):
        def put(a, tdt=None):
            t = torch.zeros(len(a) + shift, dtype=tdt or torch.from_numpy(a[:1]).dtype, device=cuda_dev)
            t[shift:] = _t(cuda_dev, a).to(t.dtype)
            return t[shift:]
        tr, tc, to, tv = put(row), put(col), put(off), put(val, dt)
        if shift:
            assert tr.data_ptr() % 16 and to.data_ptr() % 16 and tv.data_ptr() % 16
        for fn, idx in ((D.damn_spmv_coo32, tc), (D.damn_spmv_dacoo16, to)):
            y = torch.full((n,), float("nan"), dtype=dt, device=cuda_dev)
            fn(n, tr, idx, tv, tx, y)
            outs.append(y.double().cpu().numpy())
    torch.cuda.synchronize()
    for y in outs:
        assert np.array_equal(y, ref)
