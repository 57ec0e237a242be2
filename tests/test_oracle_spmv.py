"""Pins of the SpMV oracle (Section 4, Listing 2, Remark 3): hand-worked
values, exact arithmetic, the dense product, the componentwise error bound,
and sensitivity to planted mistakes."""
import numpy as np
import pytest

import workloads as W
from oracle import c_listing2 as C
from oracle import dacsr as D
from oracle import spmv as S


def _random_csr(rng, nr, nc, density=0.2, empty_rows=True):
    mask = rng.random((nr, nc)) < density
    if empty_rows:
        mask[rng.integers(0, nr, size=max(1, nr // 10))] = False
    rows, cols = np.nonzero(mask)
    vals = rng.standard_normal(len(rows))
    return W.from_coo(nr, rows, cols, vals)


def _dense(nr, nc, rp, c, v):
    A = np.zeros((nr, nc))
    for r in range(nr):
        for i in range(rp[r], rp[r + 1]):
            A[r, c[i]] += v[i]
    return A


def test_example1_by_hand():
    rp, c, v = W.example1_pattern()             # values 1..5
    x = np.array([1.0, 2.0, 3.0, 4.0])
    off = D.translate(4, rp, c)
    expect = [1.0 * 1, 2.0 * 3, 3.0 * 2 + 4.0 * 4, 5.0 * 4]
    assert S.spmv(4, rp, c, v, x, diagonal_addressed=False).tolist() == expect
    assert S.spmv(4, rp, off, v, x).tolist() == expect
    assert S.spmv_rows(4, rp, off, v, x).tolist() == expect
    # alpha, beta: y <- 2 A x - 1 y
    y = np.array([1.0, 1.0, 1.0, 1.0])
    assert S.spmv(4, rp, off, v, x, y, 2.0, -1.0).tolist() == [2 * e - 1 for e in expect]


@pytest.mark.parametrize("seed", range(6))
def test_row_loop_equals_vectorised(seed):
    rng = np.random.default_rng(seed)
    nr, nc = int(rng.integers(1, 60)), int(rng.integers(1, 60))
    rp, c, v = _random_csr(rng, nr, nc)
    off = D.translate(nr, rp, c)
    x = rng.standard_normal(nc)
    y = rng.standard_normal(nr)
    for a, b in [(1.0, 0.0), (-1.5, 0.25)]:
        for dt in (np.float64, np.float32):
            r1 = S.spmv_rows(nr, rp, off, v, x, y, a, b, dtype=dt)
            r2 = S.spmv(nr, rp, off, v, x, y, a, b, dtype=dt)
            r3 = S.spmv(nr, rp, c, v, x, y, a, b, diagonal_addressed=False, dtype=dt)
            assert np.array_equal(r1, r2) and np.array_equal(r2, r3)


@pytest.mark.parametrize("seed", range(6))
def test_dense_and_exact_within_bound(seed):
    rng = np.random.default_rng(10 + seed)
    nr, nc = int(rng.integers(1, 50)), int(rng.integers(1, 50))
    rp, c, v = _random_csr(rng, nr, nc, density=0.3)
    off = D.translate(nr, rp, c)
    x = rng.standard_normal(nc)
    y = rng.standard_normal(nr)
    A = _dense(nr, nc, rp, c, v)
    for a, b in [(1.0, 0.0), (0.75, -2.0)]:
        got = S.spmv(nr, rp, off, v, x, y, a, b)
        ex = S.spmv_exact(nr, rp, off, v, x, y, a, b)
        bnd = S.error_bound(nr, rp, off, v, x, y, a, b)
        assert np.all(np.abs(got - ex) <= bnd)
        dense = a * (A @ x) + (b * y if b != 0 else 0.0)
        assert np.all(np.abs(dense - ex) <= 2 * bnd)


def test_dyadic_is_exact():
    rp, c, v = W.laplace2d_5pt(64)
    n = 64 * 64
    x = W.dyadic_vector(n, W.rng_for(1, 1))
    off = D.translate(n, rp, c)
    got = S.spmv(n, rp, off, v, x)
    assert np.array_equal(got, S.spmv_exact(n, rp, off, v, x))
    # also exact in FP32: every partial sum is a multiple of 2^-20 below 2^3
    got32 = S.spmv_lowp(n, rp, off, v, x.astype(np.float32))
    assert np.array_equal(got32.astype(np.float64), got)


def test_beta_zero_ignores_y_and_empty_rows():
    rp = np.array([0, 2, 2, 3], dtype=np.int32)
    c = np.array([0, 2, 1], dtype=np.int32)
    v = np.array([1.0, 2.0, 3.0])
    x = np.array([1.0, 1.0, 1.0])
    y = np.array([np.nan, np.inf, np.nan])
    out = S.spmv(3, rp, c, v, x, y, 1.0, 0.0, diagonal_addressed=False)
    assert out.tolist() == [3.0, 0.0, 3.0]
    out = S.spmv(3, rp, c, v, x, np.array([1.0, 5.0, 1.0]), 1.0, 2.0, diagonal_addressed=False)
    assert out.tolist() == [5.0, 10.0, 5.0]


def test_tall_matrix_remark3():
    # nrows > ncols: x shifted by the row points outside x but is only read
    # at in-range columns
    rp, c, v = W.from_coo(6, [0, 3, 5, 5], [0, 1, 0, 2], [1.0, 2.0, 3.0, 4.0])
    off = D.translate(6, rp, c)
    x = np.array([10.0, 20.0, 30.0])
    assert S.spmv(6, rp, off, v, x).tolist() == [10.0, 0.0, 0.0, 40.0, 0.0, 150.0]


@pytest.mark.parametrize("nthreads", [1, 3])
def test_c_listing2_bitwise(nthreads):
    rng = np.random.default_rng(7)
    n = 3000
    rp, c, v = W.random_banded(n, 100, rng)
    off = D.translate(n, rp, c).astype(np.int16)
    x = rng.uniform(-1, 1, n)
    y = rng.standard_normal(n)
    for a, b in [(1.0, 0.0), (-0.5, 1.25)]:
        ref = S.spmv(n, rp, off, v, x, y, a, b)
        assert np.array_equal(C.spmv_dacsr16(n, rp, off, v, x, y, a, b, nthreads), ref)
        assert np.array_equal(C.spmv_csr32(n, rp, c, v, x, y, a, b, nthreads), ref)


def test_round_to_bf16_by_hand():
    one = 1.0
    cases = [
        (1.0, 1.0),
        (1 + 2 ** -8, 1.0),                    # halfway, tie to even (down)
        (1 + 3 * 2 ** -8, 1 + 2 ** -6),        # halfway, tie to even (up)
        (1 + 2 ** -8 + 2 ** -40, 1 + 2 ** -7),  # just above halfway: one rounding, not two
        (-(1 + 2 ** -7), -(1 + 2 ** -7)),
        (26.5, 26.5),
        (0.1, 0.10009765625),
        (2.0 ** -133, 2.0 ** -133),             # smallest bf16 subnormal
        (2.0 ** -135, 0.0),
        (3.4e38, np.inf),
    ]
    got = S.round_to_bf16([a for a, _ in cases])
    assert got.tolist() == [b for _, b in cases]


def test_round_to_bf16_matches_torch_on_fp32_inputs():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000),
                        rng.standard_normal(1000) * 1e-39]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.round_to_bf16(v.astype(np.float64)), ref)


def test_lowp_spmv_bound():
    rng = np.random.default_rng(5)
    n = 500
    rp, c, v = W.random_banded(n, 30, rng)
    off = D.translate(n, rp, c)
    x32 = rng.uniform(-1, 1, n).astype(np.float32)
    for q in ("f32", "bf16"):
        vq = S.quantize(v, q)
        got = S.spmv_lowp(n, rp, off, vq, x32)
        ex = S.spmv_exact(n, rp, off, vq, x32.astype(np.float64))
        bnd = S.error_bound(n, rp, off, vq, x32, u=S.U32)
        assert np.all(np.abs(got - ex) <= bnd)
        # quantisation error of the values against the FP64 matrix
        ex64 = S.spmv_exact(n, rp, off, v, x32.astype(np.float64))
        u_v = S.U32 if q == "f32" else S.UBF16
        tot = bnd + u_v * S.abs_row_sums(n, rp, off, v, x32)
        assert np.all(np.abs(got - ex64) <= tot)


def test_spmm_columns():
    rng = np.random.default_rng(9)
    n = 200
    rp, c, v = W.random_banded(n, 20, rng)
    off = D.translate(n, rp, c)
    X = rng.uniform(-1, 1, (n, 4))
    Y = S.spmm(n, rp, off, v, X)
    A = _dense(n, n, rp, c, v)
    for j in range(4):
        assert np.array_equal(Y[:, j], S.spmv(n, rp, off, v, X[:, j]))
    bnd = np.stack([S.error_bound(n, rp, off, v, X[:, j]) for j in range(4)], 1)
    assert np.all(np.abs(Y - A @ X) <= 2 * bnd)


@pytest.mark.parametrize("mistake", ["index_sign", "dropped_term", "transposed", "value_sign",
                                     "beta_ignored"])
def test_planted_mistakes_are_caught(mistake, monkeypatch):
    """Each plausible slip in the oracle breaks the dense-product check."""
    rng = np.random.default_rng(11)
    nr = nc = 40
    rp, c, v = _random_csr(rng, nr, nc, density=0.25, empty_rows=False)
    off = D.translate(nr, rp, c)
    x = rng.standard_normal(nc)
    y = rng.standard_normal(nr)
    A = _dense(nr, nc, rp, c, v)
    a, b = 1.5, 0.5
    if mistake == "index_sign":
        monkeypatch.setattr(S, "_columns",
                            lambda n, p, i, da: (D.entry_rows(n, p) - np.asarray(i, dtype=np.int64)) % nc)
        got = S.spmv(nr, rp, off, v, x, y, a, b)
    elif mistake == "dropped_term":
        rp_short = rp.copy()
        got = np.zeros(nr)
        for r in range(nr):
            got[r] = a * sum(v[i] * x[c[i]] for i in range(rp_short[r], rp_short[r + 1] - 1)) + b * y[r]
    elif mistake == "transposed":
        rpT, cT, vT = W.from_coo(nc, c, D.entry_rows(nr, rp), v)
        got = S.spmv(nc, rpT, cT, vT, x, y, a, b, diagonal_addressed=False)
    elif mistake == "value_sign":
        got = S.spmv(nr, rp, off, -v, x, y, a, b)
    else:
        got = S.spmv(nr, rp, off, v, x, y, a, 0.0)
    dense = a * (A @ x) + b * y
    bnd = S.error_bound(nr, rp, off, v, x, y, a, b)
    assert np.any(np.abs(got - dense) > 2 * bnd)


# --------------------------------------------------------------------------
# error_bound: exact values on a hand-worked matrix.  The tolerance of every
# random-input GPU test is this function, so it is pinned to the formula of
# the componentwise bound written out with the numbers of a small example:
#
#   alpha = 1, beta = 0:  4 * len * u * S + len * tiny
#   otherwise:            4 * (len + 2) * u * (|alpha| S + |beta| |y0|) + (len + 2) * tiny
#
# with S = sum_j |a_rj x_j|, len the row's stored entries, u the unit
# roundoff of the accumulation type and tiny its smallest normal number.
# --------------------------------------------------------------------------
TINY64 = 2.0 ** -1022
TINY32 = 2.0 ** -126


def _bound_example():
    # 3 x 4 matrix, row 1 empty:
    #   row 0: a = (1 at col 0, -2 at col 2)             S = |1*3| + |-2*0.5|          = 4,    len 2
    #   row 2: a = (0.25 at col 1, 8 at col 2, -1 at col 3)
    #                                        S = |0.25*5| + |8*0.5| + |-1*-4| = 9.25, len 3
    rp = np.array([0, 2, 2, 5], dtype=np.int32)
    col = np.array([0, 2, 1, 2, 3], dtype=np.int32)
    val = np.array([1.0, -2.0, 0.25, 8.0, -1.0])
    x = np.array([3.0, 5.0, 0.5, -4.0])
    y0 = np.array([2.0, -1.0, 0.5])
    return rp, col, val, x, y0


def _bound_pin_failures(bound_fn):
    """Cases where bound_fn differs from the hand-computed bound (empty list:
    the pin holds)."""
    rp, col, val, x, y0 = _bound_example()
    off = D.translate(3, rp, col)
    cases = []
    for u, tiny in ((S.U64, TINY64), (S.U32, TINY32)):
        # alpha = 1, beta = 0
        cases.append((dict(u=u), [4 * 2 * u * 4 + 2 * tiny, 0.0, 4 * 3 * u * 9.25 + 3 * tiny]))
        # alpha = 0.5, beta = -3, y0 = (2, -1, 0.5)
        cases.append((dict(y=y0, alpha=0.5, beta=-3.0, u=u),
                      [4 * 4 * u * (0.5 * 4 + 3 * 2) + 4 * tiny,
                       4 * 2 * u * (0.0 + 3 * 1) + 2 * tiny,
                       4 * 5 * u * (0.5 * 9.25 + 3 * 0.5) + 5 * tiny]))
        # alpha = -2, beta = 0 (general branch without the y term)
        cases.append((dict(alpha=-2.0, u=u),
                      [4 * 4 * u * (2 * 4) + 4 * tiny, 2 * tiny,
                       4 * 5 * u * (2 * 9.25) + 5 * tiny]))
    bad = []
    for kw, expect in cases:
        for idx, da in ((off, True), (col, False)):
            kw2 = dict(kw)
            got = bound_fn(3, rp, idx, val, x, kw2.pop("y", None), kw2.pop("alpha", 1.0),
                           kw2.pop("beta", 0.0), diagonal_addressed=da, **kw2)
            if not np.allclose(got, expect, rtol=1e-14, atol=0.0):
                bad.append((kw, da, list(got), expect))
    # subnormal products: S = 2^-1060 is below the normal range, the relative
    # term underflows and the absolute term len * tiny is the whole bound
    rp1 = np.array([0, 1], dtype=np.int32)
    got = bound_fn(1, rp1, np.array([0]), np.array([2.0 ** -1000]), np.array([2.0 ** -60]),
                   diagonal_addressed=False)
    if not np.allclose(got, [TINY64], rtol=1e-14, atol=0.0):
        bad.append(("subnormal", list(got), [TINY64]))
    return bad


def test_error_bound_hand_values():
    assert _bound_pin_failures(S.error_bound) == []


def _slipped(kind):
    """error_bound with one plausible slip planted (for the test below)."""
    def fn(nrows, rowptr, idx, val, x, y=None, alpha=1.0, beta=0.0,
           diagonal_addressed=True, u=S.U64):
        lens = np.diff(np.asarray(rowptr, dtype=np.int64)).astype(np.float64)
        if kind == "total_nnz":
            lens = np.full_like(lens, float(rowptr[-1]))
        s = S.abs_row_sums(nrows, rowptr, idx, val, x, diagonal_addressed)
        if kind == "abs_of_sum":
            cols = (D.entry_rows(nrows, rowptr) + np.asarray(idx)) if diagonal_addressed \
                else np.asarray(idx)
            s = np.abs(np.bincount(D.entry_rows(nrows, rowptr),
                                   weights=np.asarray(val) * np.asarray(x)[cols],
                                   minlength=nrows))
        uu = S.U32 if (kind == "u_swapped" and u == S.U64) else u
        tiny = np.finfo(np.float64 if u == S.U64 else np.float32).tiny
        if kind == "no_tiny":
            tiny = 0.0
        k = 40.0 if kind == "factor_10" else 4.0
        if alpha == 1.0 and beta == 0.0 and kind != "plus2_always":
            return k * lens * uu * s + lens * tiny
        yabs = np.abs(np.asarray(y, dtype=np.float64)) if beta != 0 else 0.0
        if kind == "beta_dropped":
            yabs = 0.0
        return k * (lens + 2.0) * uu * (abs(alpha) * s + abs(beta) * yabs) + (lens + 2.0) * tiny
    return fn


@pytest.mark.parametrize("kind", ["u_swapped", "total_nnz", "factor_10", "plus2_always",
                                  "beta_dropped", "abs_of_sum", "no_tiny"])
def test_error_bound_pin_catches_slips(kind):
    """Each slip -- a looser or a tighter bound -- fails the hand-value pin."""
    assert _bound_pin_failures(_slipped(kind)) != []


def test_error_bound_accepts_and_rejects_at_its_edge():
    """A result 8 ulps from the exact value of a row sum 2 with bound
    32 * 2^-53 = 8 ulps(2) is accepted; 9 ulps is rejected, as a GPU result
    just outside the stated tolerance must be."""
    rp, col, val, x, _ = _bound_example()
    off = D.translate(3, rp, col)
    ex = S.spmv_exact(3, rp, off, val, x)
    bnd = S.error_bound(3, rp, off, val, x)
    assert ex[0] == 2.0 and bnd[0] == 8 * np.spacing(2.0)
    y = ex.copy()
    for _ in range(8):
        y[0] = np.nextafter(y[0], np.inf)
    assert np.all(np.abs(y - ex) <= bnd)
    y[0] = np.nextafter(y[0], np.inf)
    assert not np.all(np.abs(y - ex) <= bnd)


def test_recursive_summation_error_reaches_a_quarter_of_the_bound():
    """The bound is not loose by more than its factor 4: left-to-right
    summation of 1 + u + u + ... (every partial sum rounds back to 1, ties to
    even) loses (len - 1) u, a quarter of 4 len u S up to O(1/len)."""
    n = 1001
    rp = np.array([0, n], dtype=np.int32)
    val = np.concatenate([[1.0], np.full(n - 1, S.U64)])
    x = np.ones(n)
    col = np.arange(n, dtype=np.int32)
    got = S.spmv(1, rp, col, val, x, diagonal_addressed=False)
    ex = S.spmv_exact(1, rp, col, val, x, diagonal_addressed=False)
    bnd = S.error_bound(1, rp, col, val, x, diagonal_addressed=False)
    assert got[0] == 1.0
    err = abs(got[0] - ex[0])
    assert err <= bnd[0] and err >= 0.24 * bnd[0]


def test_round_to_e4m3_by_hand():
    """E4M3 values worked out from the format: 3 significand bits, bias 7,
    largest finite 448, subnormal spacing 2^-9, no infinity."""
    cases = [
        (1.0, 1.0),
        (1 + 2 ** -4, 1.0),                    # halfway, tie to even (down)
        (1 + 3 * 2 ** -4, 1.25),               # halfway, tie to even (up)
        (1 + 2 ** -4 + 2 ** -30, 1.125),       # just above halfway: one rounding
        (-2.5, -2.5),
        (0.1, 13 * 2 ** -7),                   # 0.1 = 1.6 * 2^-4, spacing 2^-7
        (232.0, 224.0),                        # 14.5 steps of 16, tie to even
        (240.0, 240.0),
        (448.0, 448.0),                        # largest finite
        (464.0, 448.0),                        # midpoint to 480: tie to even
        (464.01, np.nan),                      # rounds to 480, not representable
        (2.0 ** -6, 2.0 ** -6),                # smallest normal
        (2.0 ** -9, 2.0 ** -9),                # smallest subnormal
        (2.0 ** -10, 0.0),                     # half of it: tie to even (zero)
        (3 * 2.0 ** -11, 2.0 ** -9),
        (7 * 2.0 ** -9, 7 * 2.0 ** -9),        # largest subnormal
        (np.inf, np.nan),
        (-0.0, -0.0),
    ]
    got = S.round_to_e4m3([a for a, _ in cases])
    want = np.array([b for _, b in cases])
    assert np.array_equal(got, want, equal_nan=True)
    assert np.signbit(got[-1])


def test_round_to_e4m3_matches_torch_on_fp32_inputs():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    rng = np.random.default_rng(8)
    v = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-4, 3, 20000),
                        rng.uniform(-500, 500, 2000), rng.uniform(-2 ** -6, 2 ** -6, 2000)])
    v = v.astype(np.float32)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(S.round_to_e4m3(v.astype(np.float64)), ref, equal_nan=True)


def test_round_to_e4m3_error_bound():
    """|fl(a) - a| <= max(2^-4 |a|, 2^-10) for every finite a up to 448: the
    per-value error used for the FP8 SpMV tolerance."""
    rng = np.random.default_rng(9)
    a = np.concatenate([rng.standard_normal(50000) * 10.0 ** rng.integers(-5, 3, 50000),
                        rng.uniform(-448, 448, 5000)])
    q = S.round_to_e4m3(a)
    assert np.all(np.abs(q - a) <= np.maximum(S.UF8 * np.abs(a), S.F8_TINY_ABS))
