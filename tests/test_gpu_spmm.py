"""GPU multi-RHS SpMM (single matrix and batched persistent launch) against
the oracle: every column within the componentwise bound of the exact product;
batched == per-matrix results bitwise; graph replay == direct launch."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import dacsr as OD
from oracle import spmv as OS

pytestmark = pytest.mark.gpu


def _t(dev, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _lanes(k):
    L = 1
    while L * 2 <= min(k, 32):
        L *= 2
    return L


def _entry_lanes(nrows, nnz, L):
    """The single-matrix call's choice: about four entries per lane and pass."""
    avg = nnz / nrows if nrows else 0.0
    E = 1
    while E * 2 * L <= 32 and E * 2 * 4 <= avg:
        E *= 2
    return E


def _check_cols(n, rp, off, val, X, Y, u):
    """Every column against the oracle's FP64 product (both within their own
    bounds of the exact result); the first and last column against the exact
    rational product itself."""
    X = X.astype(np.float64)
    ref = OS.spmm(n, rp, off, val, X)
    for j in range(X.shape[1]):
        b_gpu = OS.error_bound(n, rp, off, val, X[:, j], u=u)
        b_ref = OS.error_bound(n, rp, off, val, X[:, j], u=OS.U64)
        assert np.all(np.abs(Y[:, j] - ref[:, j]) <= b_gpu + b_ref), j
    for j in sorted({0, X.shape[1] - 1}):
        ex = OS.spmv_exact(n, rp, off, val, X[:, j])
        assert np.all(np.abs(Y[:, j] - ex) <= OS.error_bound(n, rp, off, val, X[:, j], u=u)), j


@pytest.mark.parametrize("k", [1, 3, 4, 16, 33])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_spmm_single(D, cuda_dev, k, dt):
    rng = np.random.default_rng(k)
    n = 2500
    rp, col, val = W.random_banded(n, 300, rng)
    off = OD.translate(n, rp, col)
    npd = np.float64 if dt == torch.float64 else np.float32
    valq = val.astype(npd).astype(np.float64)
    X = W.uniform_block(n, k, rng, npd)
    Y = torch.full((n, k), float("nan"), dtype=dt, device=cuda_dev)
    D.damn_spmm_dacsr16(_t(cuda_dev, rp), _t(cuda_dev, off.astype(np.int16)), _t(cuda_dev, val).to(dt),
                        _t(cuda_dev, X), Y)
    torch.cuda.synchronize()
    _check_cols(n, rp, off, valq, X, Y.double().cpu().numpy(), OS.U64 if dt == torch.float64 else OS.U32)


@pytest.mark.parametrize("k", [1, 4, 16])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_batched_matches_single_and_oracle(D, cuda_dev, k, dt):
    mats_np = W.batch_banded(12, seed=99, n_median=3000, n_min=1000, n_max=20000)
    rng = np.random.default_rng(5)
    mats, ref = [], []
    for n, rp, col, val in mats_np:
        off = OD.translate(n, rp, col).astype(np.int16)
        X = W.uniform_block(n, k, rng, np.float64 if dt == torch.float64 else np.float32)
        tv = _t(cuda_dev, val).to(dt)
        Y = torch.full((n, k), float("nan"), dtype=dt, device=cuda_dev)
        mats.append((_t(cuda_dev, rp), _t(cuda_dev, off), tv, _t(cuda_dev, X), Y))
        ref.append((n, rp, off, val, X))
    plan = D.BatchPlan(mats, k, dt, autotune=True)
    desc = plan.describe()
    assert desc["graph_ready"] == 1 and desc["count"] == 12
    plan.launch()
    torch.cuda.synchronize()
    direct = [m[4].clone() for m in mats]
    for m in mats:
        m[4].fill_(float("nan"))
    plan.graph_launch()
    torch.cuda.synchronize()
    E = desc["entry_lanes"]
    L = _lanes(k)
    assert E >= 1 and L * E <= 32
    for (rp, off, tv, tX, Y), d0 in zip(mats, direct):
        assert torch.equal(Y, d0)
        Ys = torch.empty_like(Y)
        D.damn_spmm_dacsr16(rp, off, tv, tX, Ys)
        torch.cuda.synchronize()
        if _entry_lanes(rp.numel() - 1, off.numel(), L) == E:
            assert torch.equal(Ys, Y)   # same summation shape (k, E): same bits
        else:
            scale = Y.abs().max().item() + 1.0
            tol = 1e-12 if dt == torch.float64 else 1e-4
            assert torch.allclose(Ys, Y, rtol=0, atol=tol * scale)
    u = OS.U64 if dt == torch.float64 else OS.U32
    for (n, rp, off, val, X), (_, _, tv, _, Y) in zip(ref[:4], mats[:4]):
        valq = val.astype(np.float32).astype(np.float64) if dt == torch.float32 else val
        _check_cols(n, rp, off.astype(np.int64), valq, X, Y.double().cpu().numpy(), u)


def test_batched_empty_and_k1_equals_spmv(D, cuda_dev):
    plan = D.BatchPlan([], 1, torch.float64, autotune=False)
    plan.launch()
    plan.graph_launch()
    n = 4096
    rp, col, val = W.laplace2d_5pt(64)
    off = OD.translate(n, rp, col)
    x = W.dyadic_vector(n, W.rng_for(1, 1))
    Y = torch.empty((n, 1), dtype=torch.float64, device=cuda_dev)
    D.damn_spmm_dacsr16(_t(cuda_dev, rp), _t(cuda_dev, off.astype(np.int16)), _t(cuda_dev, val),
                        _t(cuda_dev, x.reshape(n, 1)), Y)
    torch.cuda.synchronize()
    assert np.array_equal(Y.cpu().numpy()[:, 0], OS.spmv(n, rp, off, val, x))
