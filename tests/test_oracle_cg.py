"""Pins of the CG / CG-IR oracle: dense solves, the closed-form spectrum of the
27-point stencil, the CG iteration bound and the true residual."""
import numpy as np
import pytest

import workloads as W
from oracle import cg as G
from oracle import dacsr as D
from oracle import spmv as S


def _dense(n, rp, c, v):
    A = np.zeros((n, n))
    for r in range(n):
        A[r, c[rp[r]:rp[r + 1]]] = v[rp[r]:rp[r + 1]]
    return A


def test_stencil27_spectrum_closed_form():
    m = 5
    rp, c, v = W.stencil27(m)
    A = _dense(m ** 3, rp, c, v)
    lam = np.linalg.eigvalsh(A)
    lo, hi = G.stencil27_eigen_extremes(m)
    assert abs(lam[0] - lo) < 1e-10 and abs(lam[-1] - hi) < 1e-10
    lo160, hi160 = G.stencil27_eigen_extremes(160)
    assert 0.5 < lo160 < 0.52 and 36.4 < hi160 < 36.5   # kappa ~ 72


def test_cg_matches_dense_solve():
    m = 16
    rp, c, v = W.laplace2d_5pt(m)
    n = m * m
    off = D.translate(n, rp, c)
    rng = np.random.default_rng(0)
    xs = rng.uniform(-1, 1, n)
    A = _dense(n, rp, c, v)
    b = A @ xs
    res = G.cg(n, rp, off, v, b, rtol=1e-10)
    assert res.converged
    lam = np.linalg.eigvalsh(A)
    kappa = lam[-1] / lam[0]
    x_ref = np.linalg.solve(A, b)
    assert np.linalg.norm(res.x - x_ref) <= 10 * kappa * 1e-10 * np.linalg.norm(x_ref)
    # the recurrence residual is close to the true one
    true = np.linalg.norm(b - A @ res.x) / np.linalg.norm(b)
    assert true <= 1e-9
    # classical bound: iterations <= 1/2 sqrt(kappa) ln(2/tol)
    assert res.iterations <= 0.5 * np.sqrt(kappa) * np.log(2 / 1e-10) + 1


@pytest.mark.parametrize("lowp", ["f32", "bf16"])
def test_cg_ir_reaches_fp64_accuracy(lowp):
    m = 10
    rp, c, v = W.stencil27(m)
    n = m ** 3
    off = D.translate(n, rp, c)
    rng = W.rng_for(4, 1)
    xs = W.uniform_vector(n, rng)
    b = S.spmv(n, rp, off, v, xs)
    vq = S.quantize(v, lowp)
    assert np.array_equal(vq, v)  # 26.5 and -1 are exact in FP32 and BF16
    res = G.cg_ir(n, rp, off, v, vq, b, rtol=1e-10, inner_rtol=1e-3 if lowp == "f32" else 1e-2)
    assert res.converged and res.relres <= 1e-10
    r = b - S.spmv(n, rp, off, v, res.x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    lo, hi = G.stencil27_eigen_extremes(m)
    assert np.linalg.norm(res.x - xs) <= (hi / lo) * 1e-10 * np.linalg.norm(xs) * 2
    # several outer steps were needed: one FP32 inner solve alone is not enough
    assert res.outer >= 2


def test_cg_ir_with_quantised_values():
    """Perturbed off-diagonals make the BF16 copy differ from the FP64 matrix;
    refinement still reaches the FP64 tolerance."""
    m = 8
    rp, c, v = W.stencil27(m)
    n = m ** 3
    rng = np.random.default_rng(4)
    # symmetric perturbation of the off-diagonals (A stays SPD, diagonally dominant)
    A = _dense(n, rp, c, v)
    P = np.triu(rng.normal(0, 0.01, (n, n)) * (A != 0), 1)
    A = A + P + P.T
    v2 = np.array([A[r, c[i]] for r in range(n) for i in range(rp[r], rp[r + 1])])
    off = D.translate(n, rp, c)
    b = A @ rng.uniform(-1, 1, n)
    vq = S.quantize(v2, "bf16")
    assert not np.array_equal(vq, v2)
    res = G.cg_ir(n, rp, off, v2, vq, b, rtol=1e-10, inner_rtol=1e-2)
    assert res.converged
    assert np.linalg.norm(b - A @ res.x) <= 1.5e-10 * np.linalg.norm(b)


def test_inner_cg_finite_termination_on_a_diagonal_matrix():
    """CG ends after as many steps as the matrix has distinct eigenvalues
    (exact arithmetic).  On diag(2, 4, ..., 2, 4) with FP32 vectors the inner
    solve reaches d = s / diag to FP32 accuracy in two steps, and a third is
    never needed; a zero right-hand side takes no step."""
    n = 64
    rowptr = np.arange(n + 1, dtype=np.int32)
    off = np.zeros(n, dtype=np.int16)                  # DA-CSR: the diagonal
    diag = np.where(np.arange(n) % 2 == 0, 2.0, 4.0).astype(np.float32)
    s = np.random.default_rng(3).uniform(-1, 1, n).astype(np.float32)
    d, it = G.cg_lowp(n, rowptr, off, diag, s, inner_rtol=1e-6, max_inner=10)
    assert it == 2
    assert d.dtype == np.float32
    np.testing.assert_allclose(d, s / diag, rtol=1e-5, atol=1e-7)
    d0, it0 = G.cg_lowp(n, rowptr, off, diag, np.zeros(n, dtype=np.float32), max_inner=10)
    assert it0 == 0 and not d0.any()
    # one distinct eigenvalue: one step
    d1, it1 = G.cg_lowp(n, rowptr, off, np.full(n, 2.0, dtype=np.float32), s,
                        inner_rtol=1e-6, max_inner=10)
    assert it1 == 1
    np.testing.assert_allclose(d1, s / 2.0, rtol=1e-6)
