"""DA-CSR-8 (int8 offsets; the int8 index width of Section 2, Fig. 3)
through the C ABI: conversion and fit check bit-exact with the oracle, and
SpMV bitwise equal to DA-CSR-16 and CSR-32 under one plan, bitwise equal to
the oracle on dyadic inputs, within the error bound otherwise."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import dacsr as OD
from oracle import spmv as OS

pytestmark = pytest.mark.gpu


def _t(dev, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("extreme,fits", [(127, True), (-128, True), (128, False), (-129, False)])
def test_convert8_boundary(D, cuda_dev, extreme, fits):
    n = 5000
    r = 2500
    rows = np.append(np.arange(n), r)
    cols = np.append(np.arange(n), r + extreme)
    rp, c, _ = W.from_coo(n, rows, cols)
    off, info = D.damn_csr_to_dacsr8(_t(cuda_dev, rp), _t(cuda_dev, c), n)
    ref_off, ref = OD.to_dacsr8(n, n, rp, c)
    assert (info.fits, info.w, info.min_off, info.max_off, info.n_fit, info.n_bad) == \
        (ref.fits, ref.w, ref.min_off, ref.max_off, ref.n_fit, ref.n_bad)
    if fits:
        assert np.array_equal(off.cpu().numpy(), ref_off)


def test_convert8_nofit_raises(D, cuda_dev):
    rp, c, _ = W.laplace2d_5pt(128)                    # w = 128: no int8 fit
    with pytest.raises(D.DamnError):
        D.damn_csr_to_dacsr8(_t(cuda_dev, rp), _t(cuda_dev, c), 128 * 128, raise_on_nofit=True)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("tiling", [None, "rows", "slices"])
def test_spmv8_matches_16_and_32(D, cuda_dev, dt, tiling):
    rng = np.random.default_rng(8)
    n = 20000
    rp, col, val = W.random_banded(n, 100, rng)      # half-bandwidth 100 < 128
    off8, info = D.damn_csr_to_dacsr8(_t(cuda_dev, rp), _t(cuda_dev, col), n, raise_on_nofit=True)
    off16, _ = D.damn_csr_to_dacsr(_t(cuda_dev, rp), _t(cuda_dev, col), n, raise_on_nofit=True)
    t_rp, t_col = _t(cuda_dev, rp), _t(cuda_dev, col)
    t_val = _t(cuda_dev, val).to(dt) if dt != torch.bfloat16 else \
        D.damn_cast_values(_t(cuda_dev, val), torch.bfloat16)
    vec = torch.float64 if dt == torch.float64 else torch.float32
    x = _t(cuda_dev, W.uniform_vector(n, rng)).to(vec)
    plan = D.Plan(t_rp, len(col), n, dt, idx=off8)
    if tiling:
        plan.set_tiling({"rows": D.DAMN_TILING_ROWS, "slices": D.DAMN_TILING_SLICES}[tiling])
    ys = []
    for fn, idx in ((D.damn_spmv_dacsr8, off8), (D.damn_spmv_dacsr16, off16),
                    (D.damn_spmv_csr32, t_col)):
        y = torch.full((n,), float("nan"), dtype=vec, device=cuda_dev)
        fn(t_rp, idx, t_val, x, y, plan=plan)
        ys.append(y)
    torch.cuda.synchronize()
    assert torch.equal(ys[0], ys[1]) and torch.equal(ys[0], ys[2])
    if dt == torch.float64:
        off = OD.translate(n, rp, col)
        xs = x.cpu().numpy()
        rows = np.arange(0, n, 97)
        ex = OS.spmv_exact(n, rp, off, val, xs, rows=rows)
        bnd = OS.error_bound(n, rp, off, val, xs)[rows]
        assert np.all(np.abs(ys[0].cpu().numpy()[rows] - ex) <= bnd)
    assert D.damn_device_status(reset=True) == D.DAMN_OK


def test_spmv8_dyadic_bitwise_oracle(D, cuda_dev):
    m = 100
    n = m * m
    rp, col, val = W.laplace2d_5pt(m)                 # w = 100: fits int8
    x = W.dyadic_vector(n, W.rng_for(1, 1))
    off8, _ = D.damn_csr_to_dacsr8(_t(cuda_dev, rp), _t(cuda_dev, col), n, raise_on_nofit=True)
    y = torch.empty(n, dtype=torch.float64, device=cuda_dev)
    D.damn_spmv_dacsr8(_t(cuda_dev, rp), off8, _t(cuda_dev, val), _t(cuda_dev, x), y)
    torch.cuda.synchronize()
    off = OD.translate(n, rp, col)
    assert np.array_equal(y.cpu().numpy(), OS.spmv(n, rp, off, val, x))
