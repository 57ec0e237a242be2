"""DA-BSR (diagonal addressing applied to block CSR) through the C ABI: the
block pattern's offsets from the conversion, SpMV bitwise equal across
BSR-32 / DA-BSR-16 / DA-BSR-8, bitwise equal to the oracle on dyadic inputs
and within the error bound of the exact product otherwise."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import bsr as OB
from oracle import dacsr as OD
from oracle import spmv as OS

pytestmark = pytest.mark.gpu


def _t(dev, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _setup(D, dev, m, b, dyadic, dt=torch.float64):
    rng = np.random.default_rng(100 + b)
    nbr, browptr, bcol, bval = W.block_stencil3d(m, b, rng)
    if dyadic:
        bval = np.round(bval * 4) / 4                    # quarters: exact products and sums
    n = nbr * b
    x = W.dyadic_vector(n, rng) if dyadic else W.uniform_vector(n, rng)
    t_bp, t_bc = _t(dev, browptr), _t(dev, bcol)
    off16, fi = D.damn_csr_to_dacsr(t_bp, t_bc, nbr, raise_on_nofit=True)
    off8, fi8 = D.damn_csr_to_dacsr8(t_bp, t_bc, nbr, raise_on_nofit=True)
    assert fi.w == OD.bandwidth(nbr, browptr, bcol) == fi8.w
    tv = _t(dev, bval.reshape(-1)).to(dt) if dt != torch.bfloat16 else \
        D.damn_cast_values(_t(dev, bval.reshape(-1)), torch.bfloat16)
    vec = torch.float64 if dt == torch.float64 else torch.float32
    return dict(nbr=nbr, b=b, n=n, browptr=browptr, bcol=bcol, bval=bval, x=x, t_bp=t_bp, t_bc=t_bc,
                off16=off16, off8=off8, tv=tv, tx=_t(dev, x).to(vec), vec=vec)


def _all3(D, S, alpha=1.0, beta=0.0, y0=None):
    out = []
    for fn, idx in ((D.damn_spmv_bsr32, S["t_bc"]), (D.damn_spmv_dabsr16, S["off16"]),
                    (D.damn_spmv_dabsr8, S["off8"])):
        y = y0.clone() if y0 is not None else \
            torch.full((S["n"],), float("nan"), dtype=S["vec"], device=S["t_bp"].device)
        fn(S["t_bp"], idx, S["tv"], S["b"], S["tx"], y, alpha=alpha, beta=beta)
        out.append(y)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("b", [2, 3, 4])
def test_dabsr_dyadic_bitwise(D, cuda_dev, b):
    S = _setup(D, cuda_dev, 6, b, dyadic=True)
    ys = _all3(D, S)
    assert torch.equal(ys[0], ys[1]) and torch.equal(ys[0], ys[2])
    rp, col, val = OB.expand(S["nbr"], b, S["browptr"], S["bcol"], S["bval"])
    ref = OS.spmv(S["n"], rp, col, val, S["x"], diagonal_addressed=False)
    assert np.array_equal(ys[1].cpu().numpy(), ref)


@pytest.mark.parametrize("b", [1, 3, 8])
def test_dabsr_random_within_bound(D, cuda_dev, b):
    S = _setup(D, cuda_dev, 5, b, dyadic=False)
    ys = _all3(D, S)
    assert torch.equal(ys[0], ys[1]) and torch.equal(ys[0], ys[2])
    rp, col, val = OB.expand(S["nbr"], b, S["browptr"], S["bcol"], S["bval"])
    rows = np.arange(0, S["n"], 7)
    ex = OS.spmv_exact(S["n"], rp, col, val, S["x"], diagonal_addressed=False, rows=rows)
    bnd = OS.error_bound(S["n"], rp, col, val, S["x"], diagonal_addressed=False)[rows]
    assert np.all(np.abs(ys[1].cpu().numpy()[rows] - ex) <= bnd)


def test_dabsr_alpha_beta(D, cuda_dev):
    S = _setup(D, cuda_dev, 4, 3, dyadic=False)
    rng = np.random.default_rng(3)
    y0 = rng.uniform(-1, 1, S["n"])
    ys = _all3(D, S, alpha=-0.5, beta=2.0, y0=_t(cuda_dev, y0))
    assert torch.equal(ys[0], ys[1]) and torch.equal(ys[0], ys[2])
    rp, col, val = OB.expand(S["nbr"], 3, S["browptr"], S["bcol"], S["bval"])
    ex = OS.spmv_exact(S["n"], rp, col, val, S["x"], y=y0, alpha=-0.5, beta=2.0,
                       diagonal_addressed=False)
    bnd = OS.error_bound(S["n"], rp, col, val, S["x"], y=y0, alpha=-0.5, beta=2.0,
                         diagonal_addressed=False)
    assert np.all(np.abs(ys[1].cpu().numpy() - ex) <= bnd)


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_dabsr_reduced_precision(D, cuda_dev, dt):
    S = _setup(D, cuda_dev, 5, 3, dyadic=False, dt=dt)
    ys = _all3(D, S)
    assert torch.equal(ys[0], ys[1]) and torch.equal(ys[0], ys[2])
    rp, col, val = OB.expand(S["nbr"], 3, S["browptr"], S["bcol"], S["bval"])
    vq = OS.quantize(val, "f32" if dt == torch.float32 else "bf16")
    x32 = S["x"].astype(np.float32).astype(np.float64)
    ex = OS.spmv_exact(S["n"], rp, col, vq, x32, diagonal_addressed=False)
    bnd = OS.error_bound(S["n"], rp, col, vq, x32, diagonal_addressed=False, u=OS.U32)
    assert np.all(np.abs(ys[1].double().cpu().numpy() - ex) <= bnd)


def test_dabsr_rejects_bad_block_size(D, cuda_dev):
    S = _setup(D, cuda_dev, 3, 2, dyadic=False)
    with pytest.raises(D.DamnError):
        D.damn_spmv_dabsr16(S["t_bp"], S["off16"], S["tv"], 5, S["tx"],
                            torch.empty(S["nbr"] * 5, dtype=torch.float64, device=cuda_dev),
                            nbc=S["nbr"])
