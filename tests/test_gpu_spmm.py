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


def _odd_batch(rng):
    """Matrices with the row shapes the launch shapes must all handle: empty
    rows (leading, trailing, runs), a row far longer than a slice, a matrix
    with no entries at all, short and uneven rows; dyadic values (k/8) so
    that every partial sum is exact in FP32 and FP64."""
    mats = []
    for n, kind in ((300, "ragged"), (257, "long_row"), (64, "empty"), (1000, "short"), (5, "tiny")):
        if kind == "ragged":
            lens = rng.integers(0, 40, n)
            lens[:3] = 0
            lens[-4:] = 0
            lens[100:140] = 0
        elif kind == "long_row":
            lens = rng.integers(0, 3, n)
            lens[200] = 900
        elif kind == "empty":
            lens = np.zeros(n, dtype=np.int64)
        elif kind == "short":
            lens = np.where(rng.random(n) < 0.5, 0, rng.integers(1, 3, n))
        else:
            lens = np.array([0, 7, 0, 3, 0])
        rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        col = np.concatenate([np.sort(rng.choice(n, size=int(m), replace=int(m) > n))
                              for m in lens] + [np.zeros(0, np.int64)]).astype(np.int64)
        val = rng.integers(-8, 9, size=len(col)).astype(np.float64) / 8.0
        mats.append((n, rp, col, val))
    return mats


@pytest.mark.parametrize("shape", [(1, 1, 1, 32), (1, 7, 2, 64), (1, 64, 1, 256), (1, 1024, 4, 128),
                                   (1, 256, 8, 256), (0, 64, 1, 128), (0, 7, 2, 32)])
@pytest.mark.parametrize("k", [1, 3, 16, 40, 64])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_batched_shapes_exact(D, cuda_dev, shape, k, dt):
    """Every launch shape (streamed rows, fixed passes; entry lanes, rows per
    item, threads) on exact inputs: Y equals the oracle's product bit for
    bit, each row written once (Y starts as NaN), graph replay equal to the
    direct launch."""
    streamed, rpi, E, threads = shape
    if _lanes(k) * E > 32:
        pytest.skip("row groups wider than a warp")
    rng = np.random.default_rng(1000 * k + rpi)
    npd = np.float64 if dt == torch.float64 else np.float32
    mats, ref = [], []
    for n, rp, col, val in _odd_batch(rng):
        # columns within reach of an int16 offset (every test matrix is small)
        off = OD.translate(n, rp, col).astype(np.int16)
        X = (rng.integers(-256, 257, size=(n, k)) / 256.0).astype(npd)
        Y = torch.full((n, k), float("nan"), dtype=dt, device=cuda_dev)
        mats.append((_t(cuda_dev, rp), _t(cuda_dev, off), _t(cuda_dev, val).to(dt), _t(cuda_dev, X), Y))
        ref.append(OS.spmm(n, rp, off.astype(np.int64), val, X.astype(np.float64)))
    plan = D.BatchPlan(mats, k, dt, autotune=False)
    plan.set_shape(bool(streamed), rpi, E, threads)
    desc = plan.describe()
    assert (desc["streamed"], desc["tile_items"], desc["entry_lanes"], desc["threads"]) == \
        (streamed, rpi, E, threads)
    plan.launch()
    torch.cuda.synchronize()
    for m, r in zip(mats, ref):
        assert np.array_equal(m[4].double().cpu().numpy(), r)
    direct = [m[4].clone() for m in mats]
    for m in mats:
        m[4].fill_(float("nan"))
    plan.graph_launch()
    torch.cuda.synchronize()
    for m, d0 in zip(mats, direct):
        assert torch.equal(m[4], d0)
    assert D.damn_device_status() == D.DAMN_OK


@pytest.mark.parametrize("k", [1, 4, 16])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_streamed_equals_fixed_passes(D, cuda_dev, k, dt):
    """Streamed rows and fixed passes run the same per-row arithmetic for
    the same entry lanes: the same bits on random inputs."""
    mats_np = W.batch_banded(6, seed=7, n_median=3000, n_min=500, n_max=8000)
    rng = np.random.default_rng(k)
    mats = []
    for n, rp, col, val in mats_np:
        off = OD.translate(n, rp, col).astype(np.int16)
        X = W.uniform_block(n, k, rng, np.float64 if dt == torch.float64 else np.float32)
        mats.append((_t(cuda_dev, rp), _t(cuda_dev, off), _t(cuda_dev, val).to(dt), _t(cuda_dev, X),
                     torch.full((n, k), float("nan"), dtype=dt, device=cuda_dev)))
    plan = D.BatchPlan(mats, k, dt, autotune=False)
    L = _lanes(k)
    for E in (1, 2, 4):
        if L * E > 32:
            continue
        plan.set_shape(False, 64, E, 128)
        plan.launch()
        torch.cuda.synchronize()
        fixed = [m[4].clone() for m in mats]
        for m in mats:
            m[4].fill_(float("nan"))
        plan.set_shape(True, 1024, E, 256)
        plan.graph_launch()
        torch.cuda.synchronize()
        for m, f in zip(mats, fixed):
            assert torch.equal(m[4], f), E


def test_batch_set_shape_rejects(D, cuda_dev):
    n = 64
    rp, col, val = W.laplace2d_5pt(8)
    off = OD.translate(n, rp, col).astype(np.int16)
    X = torch.zeros((n, 4), dtype=torch.float64, device=cuda_dev)
    Y = torch.zeros((n, 4), dtype=torch.float64, device=cuda_dev)
    plan = D.BatchPlan([(_t(cuda_dev, rp), _t(cuda_dev, off), _t(cuda_dev, val), X, Y)], 4,
                       torch.float64, autotune=False)
    before = plan.describe()
    for bad in ((1, 0, 1, 128), (1, 1025, 1, 128), (1, 64, 1, 96), (1, 64, 1, 512),
                (0, 64, 3, 128), (0, 64, 16, 128), (0, 64, 0, 128), (1, 64, 16, 128)):
        with pytest.raises(RuntimeError):
            plan.set_shape(bool(bad[0]), bad[1], bad[2], bad[3])
        assert plan.describe() == before
    plan.set_shape(True, 64, 2, 128)
    assert (plan.describe()["streamed"], plan.describe()["entry_lanes"]) == (1, 2)
