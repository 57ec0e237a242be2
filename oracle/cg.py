"""Conjugate gradients in FP64 and mixed-precision iterative refinement
around a reduced-precision CG.  Test infrastructure only (see
``oracle/__init__.py``).

The paper motivates DA storage for iterative solvers and multi-precision
algorithms (Section 2, the multi-precision remark; Section 3) but gives no
solver.  The solver here is textbook material, written in its usual order:

FP64 CG (Hestenes-Stiefel), starting from x0:
    r = b - A x;  p = r;  rr = r.r
    repeat until sqrt(rr) <= rtol * ||b||  or  max_iter:
        q = A p;  a = rr / (p.q);  x += a p;  r -= a q
        rr' = r.r;  p = r + (rr'/rr) p;  rr = rr'

Iterative refinement (CG-IR), FP64 outer loop:
    repeat:
        r = b - A x            (FP64 values, FP64 accumulation)
        stop if ||r|| <= rtol * ||b||  or  max_outer
        s = r / ||r||  rounded to FP32
        d = CG on A_low d = s  (FP32 vectors, reduced-precision values with
                                FP32 accumulation, dot products accumulated in
                                FP64, to inner_rtol or max_inner steps)
        x += ||r|| d           (FP64)

Readings: norms are 2-norms; the stopping test uses ||b||; inner dot products
take the FP32 vectors, form the products in FP64 (exactly) and sum in FP64;
the step lengths a and b are FP64 numbers rounded to FP32 for the FP32 vector
updates.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .spmv import spmv, spmv_lowp


@dataclass
class CGResult:
    x: np.ndarray
    iterations: int
    converged: bool
    relres: float                      # recurrence (CG) or true (CG-IR) residual ratio
    history: list = field(default_factory=list)
    outer: int = 0


def _dot64(a, b) -> float:
    return float(np.dot(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)))


def cg(nrows, rowptr, idx, val, b, x0=None, rtol=1e-10, max_iter=1000,
       diagonal_addressed=True) -> CGResult:
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(nrows) if x0 is None else np.array(x0, dtype=np.float64)

    def A(v):
        return spmv(nrows, rowptr, idx, val, v, diagonal_addressed=diagonal_addressed)

    r = b - A(x)
    p = r.copy()
    rr = _dot64(r, r)
    nb = np.sqrt(_dot64(b, b))
    hist = [np.sqrt(rr) / nb]
    it = 0
    while np.sqrt(rr) > rtol * nb and it < max_iter:
        q = A(p)
        a = rr / _dot64(p, q)
        x = x + a * p
        r = r - a * q
        rr_new = _dot64(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        hist.append(np.sqrt(rr) / nb)
    return CGResult(x, it, bool(np.sqrt(rr) <= rtol * nb), float(np.sqrt(rr) / nb), hist)


def cg_lowp(nrows, rowptr, idx, val_lowp, s32, inner_rtol=1e-3, max_inner=100,
            diagonal_addressed=True):
    """Inner solve A_low d = s with FP32 vectors and FP64 dot products, d0 = 0.
    Returns (d, iterations)."""
    f32 = np.float32
    s32 = np.asarray(s32, dtype=f32)
    d = np.zeros(nrows, dtype=f32)
    r = s32.copy()
    p = r.copy()
    rr = _dot64(r, r)
    ns = np.sqrt(_dot64(s32, s32))
    it = 0
    while np.sqrt(rr) > inner_rtol * ns and it < max_inner:
        q = spmv_lowp(nrows, rowptr, idx, val_lowp, p, diagonal_addressed=diagonal_addressed)
        a = rr / _dot64(p, q)
        d = (d + f32(a) * p).astype(f32)
        r = (r - f32(a) * q).astype(f32)
        rr_new = _dot64(r, r)
        p = (r + f32(rr_new / rr) * p).astype(f32)
        rr = rr_new
        it += 1
    return d, it


def cg_ir(nrows, rowptr, idx, val, val_lowp, b, x0=None, rtol=1e-10, inner_rtol=1e-3,
          max_inner=100, max_outer=50, diagonal_addressed=True) -> CGResult:
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(nrows) if x0 is None else np.array(x0, dtype=np.float64)
    nb = np.sqrt(_dot64(b, b))
    hist = []
    total_inner = 0
    outer = 0
    while True:
        r = spmv(nrows, rowptr, idx, val, x, b, alpha=-1.0, beta=1.0,
                 diagonal_addressed=diagonal_addressed)
        nr = np.sqrt(_dot64(r, r))
        hist.append(nr / nb)
        if nr <= rtol * nb or outer >= max_outer:
            break
        s32 = (r / nr).astype(np.float32)
        d, it = cg_lowp(nrows, rowptr, idx, val_lowp, s32, inner_rtol, max_inner,
                        diagonal_addressed)
        total_inner += it
        x = x + nr * d.astype(np.float64)
        outer += 1
    return CGResult(x, total_inner, bool(nr <= rtol * nb), float(nr / nb), hist, outer)


def stencil27_eigen_extremes(m: int, diag: float = 26.5, off: float = -1.0):
    """Closed-form extreme eigenvalues of the 27-point stencil matrix on an
    m^3 grid with Dirichlet boundary: A = (diag - off) I + off * (T (x) T (x) T)
    with T = tridiag(1, 1, 1) of order m, whose eigenvalues are
    1 + 2 cos(j pi / (m + 1)), j = 1..m."""
    t = 1.0 + 2.0 * np.cos(np.arange(1, m + 1) * np.pi / (m + 1))
    prods = np.multiply.outer(np.multiply.outer(t, t), t).ravel()
    lam = (diag - off) + off * prods
    return float(lam.min()), float(lam.max())
