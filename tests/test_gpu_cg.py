"""GPU CG (FP64) and mixed-precision CG-IR against the oracle: the solution's
true residual is recomputed by the oracle's own SpMV, the error is checked
against x* with the condition number, and iteration counts are compared with
the oracle's CG on the same system."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cg as OC
from oracle import dacsr as OD
from oracle import spmv as OS

pytestmark = pytest.mark.gpu


def _system(cuda_dev, kind, m, perturb=False):
    if kind == "lap2d":
        rp, col, val = W.laplace2d_5pt(m)
        n = m * m
        lo, hi = 8 * np.sin(np.pi / (2 * (m + 1))) ** 2, 8 * np.cos(np.pi / (2 * (m + 1))) ** 2
    else:
        rp, col, val = W.stencil27(m)
        n = m ** 3
        lo, hi = OC.stencil27_eigen_extremes(m)
    if perturb:
        rng = np.random.default_rng(4)
        # symmetric perturbation of the off-diagonals, A stays SPD
        r = OD.entry_rows(n, rp)
        key_lo = np.minimum(r, col).astype(np.int64) * n + np.maximum(r, col)
        u = np.unique(key_lo)
        pert = rng.normal(0, 0.01, len(u))
        idx = np.searchsorted(u, key_lo)
        val = val + np.where(r != col, pert[idx], 0.0)
    off = OD.translate(n, rp, col)
    xs = W.uniform_vector(n, W.rng_for(4, 1))
    b = OS.spmv(n, rp, off, val, xs)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda_dev)
    return dict(n=n, rp=rp, col=col, val=val, off=off, xs=xs, b=b, kappa=hi / lo,
                t_rp=t(rp), t_off=t(off.astype(np.int16)), t_val=t(val), t_b=t(b))


def _true_relres(S, x):
    r = S["b"] - OS.spmv(S["n"], S["rp"], S["off"], S["val"], x)
    return np.linalg.norm(r) / np.linalg.norm(S["b"])


@pytest.mark.parametrize("kind,m", [("lap2d", 64), ("st27", 24)])
def test_cg_fp64(D, cuda_dev, kind, m):
    S = _system(cuda_dev, kind, m)
    x = torch.zeros(S["n"], dtype=torch.float64, device=cuda_dev)
    plan = D.Plan(S["t_rp"], len(S["col"]), S["n"], torch.float64, idx=S["t_off"])
    res = D.damn_cg(S["t_rp"], S["t_off"], S["t_val"], S["t_b"], x, rtol=1e-10, max_iter=2000,
                    plan=plan)
    assert res["converged"], res
    xg = x.cpu().numpy()
    assert _true_relres(S, xg) <= 2e-10
    assert abs(res["true_relres"] - _true_relres(S, xg)) <= 1e-12
    assert np.linalg.norm(xg - S["xs"]) <= 4 * S["kappa"] * 1e-10 * np.linalg.norm(S["xs"])
    ref = OC.cg(S["n"], S["rp"], S["off"], S["val"], S["b"], rtol=1e-10, max_iter=2000)
    assert abs(res["iterations"] - ref.iterations) <= max(3, ref.iterations // 20)


@pytest.mark.parametrize("lowp", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("perturb", [False, True])
def test_cg_ir(D, cuda_dev, lowp, perturb):
    S = _system(cuda_dev, "st27", 20, perturb=perturb)
    low = D.damn_cast_values(S["t_val"], lowp)
    x = torch.zeros(S["n"], dtype=torch.float64, device=cuda_dev)
    p64 = D.Plan(S["t_rp"], len(S["col"]), S["n"], torch.float64, idx=S["t_off"])
    plow = D.Plan(S["t_rp"], len(S["col"]), S["n"], lowp, idx=S["t_off"])
    inner = 1e-3 if lowp == torch.float32 else 1e-2
    res = D.damn_cg_ir(S["t_rp"], S["t_off"], S["t_val"], low, S["t_b"], x, rtol=1e-10,
                       inner_rtol=inner, max_inner=200, max_outer=60, plan64=p64, plan_low=plow)
    assert res["converged"], res
    assert res["outer"] >= 2
    xg = x.cpu().numpy()
    assert _true_relres(S, xg) <= 1.5e-10
    assert np.linalg.norm(xg - S["xs"]) <= 4 * S["kappa"] * 1e-10 * np.linalg.norm(S["xs"])
    # the oracle's refinement with the same quantised values converges too,
    # in a comparable number of outer steps
    vq = OS.quantize(S["val"], "f32" if lowp == torch.float32 else "bf16")
    ref = OC.cg_ir(S["n"], S["rp"], S["off"], S["val"], vq, S["b"], rtol=1e-10, inner_rtol=inner,
                   max_inner=200, max_outer=60)
    assert ref.converged and abs(res["outer"] - ref.outer) <= 2


def test_cg_not_converged_and_zero_rhs(D, cuda_dev):
    S = _system(cuda_dev, "lap2d", 32)
    x = torch.zeros(S["n"], dtype=torch.float64, device=cuda_dev)
    res = D.damn_cg(S["t_rp"], S["t_off"], S["t_val"], S["t_b"], x, rtol=1e-12, max_iter=3)
    assert not res["converged"] and res["iterations"] == 3
    assert res["status"] == D.DAMN_ERR_NOT_CONVERGED
    zb = torch.zeros_like(S["t_b"])
    x = torch.zeros_like(S["t_b"])
    res = D.damn_cg(S["t_rp"], S["t_off"], S["t_val"], zb, x, rtol=1e-10, max_iter=10)
    assert res["converged"] and res["iterations"] == 0 and float(x.abs().max()) == 0.0
    # nonzero start: CG from x0 = x* returns at once
    x = torch.from_numpy(S["xs"]).to(cuda_dev)
    res = D.damn_cg(S["t_rp"], S["t_off"], S["t_val"], S["t_b"], x, rtol=1e-8, max_iter=10)
    assert res["converged"] and res["iterations"] <= 1
    assert D.damn_device_status() == 0


def test_cg_breakdown_reported_and_x_kept(D, cuda_dev):
    """A negative definite matrix makes p.q < 0 at the first step: CG stops
    with DAMN_ERR_NOT_CONVERGED (breakdown) without touching x and without
    hanging."""
    S = _system(cuda_dev, "lap2d", 16)
    neg = -S["t_val"]
    x0 = torch.full((S["n"],), 0.25, dtype=torch.float64, device=cuda_dev)
    x = x0.clone()
    res = D.damn_cg(S["t_rp"], S["t_off"], neg, S["t_b"], x, rtol=1e-10, max_iter=50)
    assert res["status"] == D.DAMN_ERR_NOT_CONVERGED and not res["converged"]
    assert torch.equal(x, x0)
    assert D.damn_device_status(reset=True) == D.DAMN_OK
