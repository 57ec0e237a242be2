"""Parity at the full sizes of the benchmark workloads, through the C ABI and
in the launch configurations the benchmark times (autotuned or heuristic
plans, the batched persistent launch and its CUDA graph).

The oracle cannot run a Fraction-exact product over 1e8 entries, so each
workload is checked on what it can compute:

* 160^3 27-point stencil (n = 4,096,000, nnz = 109,215,352): with x on a
  2^-20 grid (FP64) or a 2^-10 grid (FP32 / BF16 values, FP32 vectors) every
  partial sum of a row is exact (|row sum| < 2^7, products on a 2^-21 or
  2^-11 grid), so the whole y is bitwise equal to the oracle's Listing 2
  result; random x is checked on sampled rows against the exact product
  within 4 * nnz_row * 2^-53 * sum |a x|; CSR-32 == DA-CSR-16 bitwise.
* the same system solved by FP64 CG and by CG-IR with FP32 and BF16 inner
  values: the true relative residual, recomputed by the oracle's SpMV over
  the whole matrix, and the error against x* (condition number from the
  closed-form spectrum); CG's iteration count within the classical bound.
* 512 random banded matrices, k = 1 (FP64) and k = 16 (FP32): graph replay ==
  direct persistent launch bitwise for every matrix; the smallest, the
  largest and six seeded matrices checked column by column against the
  oracle's FP64 product (both within their bounds of the exact result).
* random banded n = 2e7, half-bandwidth 30000 (about 2.7e8 entries): CSR-32 ==
  DA-CSR-16 bitwise under the heuristic plan; sampled rows within the bound.
* DA-CSR-8 on the 2-D Laplacian with 131072 lines of 127 points
  (n = 16,646,144): dyadic x, whole y bitwise equal to the oracle, and
  DA-CSR-8 == DA-CSR-16 == CSR-32 bitwise.

These tests hold several GB of host and device memory and take minutes, so
the file name makes pytest collect them after the smaller GPU tests.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cg as OC
from oracle import dacsr as OD
from oracle import spmv as OS

pytestmark = pytest.mark.gpu


def _t(dev, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _sample_rows(n, rng, edge=300, inner=3000):
    return np.unique(np.concatenate([np.arange(0, min(edge, n)), np.arange(max(0, n - edge), n),
                                     rng.integers(0, n, inner)]))


def _check_sampled(rows, got, rp, off, val, x):
    """Sampled rows of an FP64 product against the exact (rational) result."""
    ex = OS.spmv_exact(len(rp) - 1, rp, off, val, x, rows=rows)
    lens = np.diff(rp.astype(np.int64))[rows].astype(np.float64)
    s = np.array([np.sum(np.abs(val[rp[r]:rp[r + 1]] * x[r + off[rp[r]:rp[r + 1]]]))
                  for r in rows])
    assert np.all(np.abs(got[rows] - ex) <= 4 * lens * OS.U64 * s)


# ----------------------------------------------------------------------------
# 160^3 27-point stencil: the mixed-precision CG system
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def stencil160(cuda_dev, D):
    m = 160
    n = m ** 3
    rp, col, val = W.stencil27(m)
    off = OD.translate(n, rp, col)
    t_rp, t_col = _t(cuda_dev, rp), _t(cuda_dev, col)
    t_off, info = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
    ref = OD.fit_check(n, n, rp, col)
    assert (info.fits, info.w, info.min_off, info.max_off) == \
        (ref.fits, ref.w, ref.min_off, ref.max_off)
    S = dict(n=n, m=m, rp=rp, off=off, val=val, t_rp=t_rp, t_col=t_col, t_off=t_off,
             t_val=_t(cuda_dev, val))
    yield S
    S.clear()
    torch.cuda.empty_cache()


def test_stencil27_160_spmv_fp64(D, cuda_dev, stencil160):
    S = stencil160
    n, nnz = S["n"], len(S["off"])
    plan = D.Plan(S["t_rp"], nnz, n, torch.float64, idx=S["t_off"])
    y = torch.full((n,), float("nan"), dtype=torch.float64, device=cuda_dev)
    yc = torch.full_like(y, float("nan"))
    # random x, under the autotuned plan the solvers use
    x = W.uniform_vector(n, W.rng_for(4, 1))
    t_x = _t(cuda_dev, x)
    plan.autotune(D.DAMN_FMT_DACSR16, S["t_off"], S["t_val"], t_x, y)
    D.damn_spmv_dacsr16(S["t_rp"], S["t_off"], S["t_val"], t_x, y, plan=plan)
    D.damn_spmv_csr32(S["t_rp"], S["t_col"], S["t_val"], t_x, yc, plan=plan)
    torch.cuda.synchronize()
    assert torch.equal(y, yc)
    rows = _sample_rows(n, np.random.default_rng(160))
    _check_sampled(rows, y.cpu().numpy(), S["rp"], S["off"], S["val"], x)
    # dyadic x: the whole vector bitwise
    xd = W.dyadic_vector(n, W.rng_for(4, 2))
    D.damn_spmv_dacsr16(S["t_rp"], S["t_off"], S["t_val"], _t(cuda_dev, xd), y, plan=plan)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), OS.spmv(n, S["rp"], S["off"], S["val"], xd))
    assert D.damn_device_status() == D.DAMN_OK


@pytest.mark.parametrize("lowp", [torch.float32, torch.bfloat16])
def test_stencil27_160_spmv_lowp_dyadic(D, cuda_dev, stencil160, lowp):
    """26.5 and -1 are exact in FP32 and BF16; with x on a 2^-10 grid every
    FP32 partial sum is exact too, so y is bitwise the oracle's."""
    S = stencil160
    n, nnz = S["n"], len(S["off"])
    low = D.damn_cast_values(S["t_val"], lowp)
    assert np.array_equal(low.double().cpu().numpy(), S["val"])
    plan = D.Plan(S["t_rp"], nnz, n, lowp, idx=S["t_off"])
    x32 = W.dyadic_vector(n, W.rng_for(4, 3), bits=10).astype(np.float32)
    t_x = _t(cuda_dev, x32)
    y = torch.full((n,), float("nan"), dtype=torch.float32, device=cuda_dev)
    yc = torch.full_like(y, float("nan"))
    plan.autotune(D.DAMN_FMT_DACSR16, S["t_off"], low, t_x, y)
    D.damn_spmv_dacsr16(S["t_rp"], S["t_off"], low, t_x, y, plan=plan)
    D.damn_spmv_csr32(S["t_rp"], S["t_col"], low, t_x, yc, plan=plan)
    torch.cuda.synchronize()
    assert torch.equal(y, yc)
    ref = OS.spmv_lowp(n, S["rp"], S["off"], OS.quantize(S["val"], "f32"), x32)
    assert np.array_equal(y.cpu().numpy(), ref)


def test_stencil27_160_cg_and_cg_ir(D, cuda_dev, stencil160):
    S = stencil160
    n, nnz = S["n"], len(S["off"])
    lo, hi = OC.stencil27_eigen_extremes(S["m"])
    kappa = hi / lo
    xs = W.uniform_vector(n, W.rng_for(4, 1))
    b = OS.spmv(n, S["rp"], S["off"], S["val"], xs)
    t_b = _t(cuda_dev, b)
    nb = np.linalg.norm(b)

    def check(x, relres_max):
        xg = x.cpu().numpy()
        r = b - OS.spmv(n, S["rp"], S["off"], S["val"], xg)
        assert np.linalg.norm(r) / nb <= relres_max
        assert np.linalg.norm(xg - xs) <= 4 * kappa * 1e-10 * np.linalg.norm(xs)

    p64 = D.Plan(S["t_rp"], nnz, n, torch.float64, idx=S["t_off"])
    x = torch.zeros(n, dtype=torch.float64, device=cuda_dev)
    res = D.damn_cg(S["t_rp"], S["t_off"], S["t_val"], t_b, x, rtol=1e-10, max_iter=2000,
                    plan=p64)
    assert res["converged"], res
    assert res["iterations"] <= 0.5 * np.sqrt(kappa) * np.log(2 / 1e-10) + 1
    check(x, 2e-10)
    for lowp, inner in ((torch.float32, 1e-3), (torch.bfloat16, 1e-2)):
        low = D.damn_cast_values(S["t_val"], lowp)
        plow = D.Plan(S["t_rp"], nnz, n, lowp, idx=S["t_off"])
        x.zero_()
        res = D.damn_cg_ir(S["t_rp"], S["t_off"], S["t_val"], low, t_b, x, rtol=1e-10,
                           inner_rtol=inner, max_inner=200, max_outer=60, plan64=p64,
                           plan_low=plow)
        assert res["converged"] and res["outer"] >= 2, res
        check(x, 1.5e-10)
        del low, plow
    assert D.damn_device_status() == D.DAMN_OK


# ----------------------------------------------------------------------------
# 512 random banded matrices in one persistent launch
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def batch512(cuda_dev, D):
    mats_np = W.batch_banded(512)
    dev_mats = []
    for n, rp, col, val in mats_np:
        t_rp = _t(cuda_dev, rp)
        off, _ = D.damn_csr_to_dacsr(t_rp, _t(cuda_dev, col), n, raise_on_nofit=True)
        dev_mats.append((n, t_rp, off, _t(cuda_dev, val)))
    out = {"np": mats_np, "dev": dev_mats}
    yield out
    out.clear()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("k,dt", [(1, torch.float64), (16, torch.float32)])
def test_batch512_full_size(D, cuda_dev, batch512, k, dt):
    mats_np, dev_mats = batch512["np"], batch512["dev"]
    npd = np.float64 if dt == torch.float64 else np.float32
    rng = np.random.default_rng(512 + k)
    Xs, mats = [], []
    for n, t_rp, off, t_val in dev_mats:
        X = W.uniform_block(n, k, rng, npd)
        Xs.append(X)
        Y = torch.full((n, k), float("nan"), dtype=dt, device=cuda_dev)
        mats.append((t_rp, off, t_val.to(dt), _t(cuda_dev, X), Y))
    plan = D.BatchPlan(mats, k, dt, autotune=True)
    assert plan.describe()["count"] == 512
    plan.launch()
    torch.cuda.synchronize()
    direct = [m[4].clone() for m in mats]
    for m in mats:
        m[4].fill_(float("nan"))
    plan.graph_launch()
    torch.cuda.synchronize()
    for m, d0 in zip(mats, direct):
        assert torch.equal(m[4], d0)
    sizes = np.array([m[0] for m in mats_np])
    pick = sorted({int(sizes.argmin()), int(sizes.argmax())}
                  | set(rng.choice(len(mats_np), 6, replace=False).tolist()))
    # the GPU result and the oracle's are each within their own bound of the
    # exact product (u of the accumulation type, plus a subnormal term)
    u = OS.U64 if dt == torch.float64 else OS.U32
    tiny = np.finfo(npd).tiny
    for i in pick:
        n, rp, col, val = mats_np[i]
        off = OD.translate(n, rp, col)
        valq = OS.quantize(val, "f64" if dt == torch.float64 else "f32")
        lens = np.diff(rp.astype(np.int64)).astype(np.float64)
        X = Xs[i].astype(np.float64)
        Y = mats[i][4].double().cpu().numpy()
        ref = OS.spmm(n, rp, off, valq, X)
        for j in range(k):
            s = OS.abs_row_sums(n, rp, off, valq, X[:, j])
            bound = 4.0 * lens * (u + OS.U64) * s + 2.0 * lens * tiny
            assert np.all(np.abs(Y[:, j] - ref[:, j]) <= bound), (i, j)
    plan.close()
    del mats, direct, plan
    torch.cuda.empty_cache()
    assert D.damn_device_status() == D.DAMN_OK


# ----------------------------------------------------------------------------
# the largest random banded matrix and the DA-CSR-8 grid
# ----------------------------------------------------------------------------

def test_random_banded_2e7_wide_band(D, cuda_dev):
    n, h = 20_000_000, 30000
    rp, col, val = W.random_banded(n, h, W.rng_for(3, 17))
    off = OD.translate(n, rp, col)
    t_rp, t_col, t_val = _t(cuda_dev, rp), _t(cuda_dev, col), _t(cuda_dev, val)
    t_off, info = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
    assert info.w <= h
    del col
    plan = D.Plan(t_rp, len(off), n, torch.float64, idx=t_off)
    x = W.uniform_vector(n, W.rng_for(3, 117))
    t_x = _t(cuda_dev, x)
    y = torch.full((n,), float("nan"), dtype=torch.float64, device=cuda_dev)
    yc = torch.full_like(y, float("nan"))
    D.damn_spmv_dacsr16(t_rp, t_off, t_val, t_x, y, plan=plan)
    D.damn_spmv_csr32(t_rp, t_col, t_val, t_x, yc, plan=plan)
    torch.cuda.synchronize()
    assert torch.equal(y, yc)
    rows = _sample_rows(n, np.random.default_rng(2007))
    _check_sampled(rows, y.cpu().numpy(), rp, off, val, x)
    del t_rp, t_col, t_val, t_off, t_x, y, yc, plan
    torch.cuda.empty_cache()
    assert D.damn_device_status() == D.DAMN_OK


def test_dacsr8_laplace2d_127_lines_full_size(D, cuda_dev):
    mx, my = 127, 131072
    rp, col, val = W.laplace2d_5pt_rect(mx, my)
    n = mx * my
    off = OD.translate(n, rp, col)
    t_rp, t_col, t_val = _t(cuda_dev, rp), _t(cuda_dev, col), _t(cuda_dev, val)
    off8, fi = D.damn_csr_to_dacsr8(t_rp, t_col, n, raise_on_nofit=True)
    assert fi.w == mx
    assert np.array_equal(off8.cpu().numpy().astype(np.int64), off)
    off16, _ = D.damn_csr_to_dacsr(t_rp, t_col, n, raise_on_nofit=True)
    plan = D.Plan(t_rp, len(off), n, torch.float64, idx=off8)
    xd = W.dyadic_vector(n, W.rng_for(3, 8))
    t_x = _t(cuda_dev, xd)
    ys = []
    for fn, idx in ((D.damn_spmv_dacsr8, off8), (D.damn_spmv_dacsr16, off16),
                    (D.damn_spmv_csr32, t_col)):
        y = torch.full((n,), float("nan"), dtype=torch.float64, device=cuda_dev)
        fn(t_rp, idx, t_val, t_x, y, plan=plan)
        ys.append(y)
    torch.cuda.synchronize()
    assert torch.equal(ys[0], ys[1]) and torch.equal(ys[0], ys[2])
    assert np.array_equal(ys[0].cpu().numpy(), OS.spmv(n, rp, off, val, xd))
    del ys, t_rp, t_col, t_val, off8, off16, t_x, plan
    torch.cuda.empty_cache()
    assert D.damn_device_status() == D.DAMN_OK
