"""GPU parity of the SpMV kernels (Section 4, Listing 2) against the oracle.

* dyadic inputs (every partial sum exact): bitwise equality with the oracle;
* random inputs: componentwise error bound against the exact (rational)
  product, 4 * nnz_row * 2^-53 * sum |a x| (alpha = 1, beta = 0) and its
  alpha/beta extension;
* CSR-32 and DA-CSR-16 results bitwise equal under one plan;
* every tiling mode (no plan, one row per thread with 256 / 128 consumers,
  balanced slices), ragged sizes, empty rows, long rows (tiles computed from
  global memory), non-square shapes, beta = 0 with NaN in y;
* reduced-precision values (FP32 / BF16, FP32 vectors and accumulation).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import dacsr as OD
from oracle import spmv as OS

pytestmark = pytest.mark.gpu

# plan variants: no plan; heuristic plan with x windows from off or from col;
# each tiling pinned (x windows from off); a plan without x windows (x gathered)
MODES = ["none", "auto", "auto_col", "rows", "rows_long", "slices", "rows_gather", "band",
         "band_col", "band_gather", "lanes4", "lanes8", "lanes16", "lanes32", "sorted",
         "sorted_col", "sorted_gather", "rows_x2", "rows_xg", "rows_long_xg", "band_xg"]


def _t(dev, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


class Mat:
    def __init__(self, D, dev, nrows, ncols, rp, col, val, dtype=torch.float64):
        self.nrows, self.ncols = nrows, ncols
        self.rp, self.col, self.val = rp, col, val
        self.off = OD.translate(nrows, rp, col)
        # DA-CSR-16 input must fit int16 (a wrapped offset addresses another column)
        assert self.off.size == 0 or (self.off.min() >= -32768 and self.off.max() <= 32767)
        self.t_rp = _t(dev, rp)
        self.t_col = _t(dev, col)
        self.t_off = _t(dev, self.off.astype(np.int16))
        self.t_val = _t(dev, val).to(dtype) if dtype in (torch.float64, torch.float32) else \
            D.damn_cast_values(_t(dev, val), dtype)
        self.dtype = dtype


def _plan(D, m, mode):
    if mode == "none":
        return None
    idx = {"auto_col": m.t_col, "band_col": m.t_col, "sorted_col": m.t_col, "rows_gather": None,
           "band_gather": None, "sorted_gather": None}.get(mode, m.t_off)
    p = D.Plan(m.t_rp, len(m.col), m.ncols, m.dtype, idx=idx)
    tiling = {"rows": D.DAMN_TILING_ROWS, "rows_long": D.DAMN_TILING_ROWS_LONG,
              "slices": D.DAMN_TILING_SLICES, "rows_gather": D.DAMN_TILING_ROWS,
              "band": D.DAMN_TILING_BAND, "band_col": D.DAMN_TILING_BAND,
              "band_gather": D.DAMN_TILING_BAND, "lanes4": D.DAMN_TILING_ROWS_LANES4,
              "lanes8": D.DAMN_TILING_ROWS_LANES8, "lanes16": D.DAMN_TILING_ROWS_LANES16,
              "lanes32": D.DAMN_TILING_ROWS_LANES32, "sorted": D.DAMN_TILING_SORTED_ROWS,
              "sorted_col": D.DAMN_TILING_SORTED_ROWS,
              "sorted_gather": D.DAMN_TILING_SORTED_ROWS,
              "rows_x2": D.DAMN_TILING_ROWS_X2}.get(mode)
    if mode == "rows_xg":
        tiling = D.DAMN_TILING_ROWS
    if mode == "rows_long_xg":
        tiling = D.DAMN_TILING_ROWS_LONG
    if mode == "band_xg":
        tiling = D.DAMN_TILING_BAND
    if tiling is not None:
        p.set_tiling(tiling)
    if mode.endswith("_xg"):
        p.set_x_staging(False)
    return p


def _run(D, m, x, y=None, alpha=1.0, beta=0.0, plan=None, fmt="da", stream=None):
    dev = m.t_rp.device
    vec = torch.float64 if m.dtype == torch.float64 else torch.float32
    t_x = _t(dev, x).to(vec)
    t_y = torch.full((m.nrows,), float("nan"), dtype=vec, device=dev) if y is None \
        else _t(dev, y).to(vec)
    if fmt == "da":
        D.damn_spmv_dacsr16(m.t_rp, m.t_off, m.t_val, t_x, t_y, alpha, beta, plan=plan, ncols=m.ncols)
    else:
        D.damn_spmv_csr32(m.t_rp, m.t_col, m.t_val, t_x, t_y, alpha, beta, plan=plan, ncols=m.ncols)
    torch.cuda.synchronize()
    return t_y.double().cpu().numpy()


@pytest.mark.parametrize("mode", MODES)
def test_config1_dyadic_bitwise(D, cuda_dev, mode):
    rp, col, val = W.laplace2d_5pt(64)
    n = 4096
    m = Mat(D, cuda_dev, n, n, rp, col, val)
    x = W.dyadic_vector(n, W.rng_for(1, 1))
    ref = OS.spmv(n, rp, m.off, val, x)
    plan = _plan(D, m, mode)
    assert np.array_equal(_run(D, m, x, plan=plan), ref)
    assert np.array_equal(_run(D, m, x, plan=plan, fmt="csr"), ref)
    # mixed precision is exact here as well (multiples of 2^-20 below 2^3)
    m32 = Mat(D, cuda_dev, n, n, rp, col, val, torch.float32)
    plan32 = _plan(D, m32, mode)
    assert np.array_equal(_run(D, m32, x, plan=plan32), ref)
    mb = Mat(D, cuda_dev, n, n, rp, col, val, torch.bfloat16)
    planb = _plan(D, mb, mode)
    assert np.array_equal(_run(D, mb, x, plan=planb), ref)
    # and with FP8 E4M3 values (4 and -1 are exact in E4M3)
    m8 = Mat(D, cuda_dev, n, n, rp, col, val, torch.float8_e4m3fn)
    plan8 = _plan(D, m8, mode)
    assert np.array_equal(_run(D, m8, x, plan=plan8), ref)


def _bound_check(m, x, got, y0=None, alpha=1.0, beta=0.0, u=OS.U64, vals=None):
    vals = m.val if vals is None else vals
    ex = OS.spmv_exact(m.nrows, m.rp, m.off, vals, x, y0, alpha, beta)
    bnd = OS.error_bound(m.nrows, m.rp, m.off, vals, x, y0, alpha, beta, u=u)
    bad = np.abs(got - ex) > bnd
    assert not bad.any(), (np.nonzero(bad)[0][:10], got[bad][:5], ex[bad][:5])


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,h,seed", [(1, 1, 0), (257, 5, 1), (3001, 100, 2), (12345, 1000, 3)])
def test_random_banded_bound_and_formats(D, cuda_dev, mode, n, h, seed):
    rng = np.random.default_rng(seed)
    rp, col, val = W.random_banded(n, h, rng)
    m = Mat(D, cuda_dev, n, n, rp, col, val)
    x = W.uniform_vector(n, rng)
    plan = _plan(D, m, mode)
    got = _run(D, m, x, plan=plan)
    _bound_check(m, x, got)
    assert np.array_equal(got, _run(D, m, x, plan=plan, fmt="csr"))


@pytest.mark.parametrize("mode", MODES)
def test_alpha_beta_and_nan_y(D, cuda_dev, mode):
    rng = np.random.default_rng(12)
    n = 5000
    rp, col, val = W.random_banded(n, 300, rng)
    m = Mat(D, cuda_dev, n, n, rp, col, val)
    x = W.uniform_vector(n, rng)
    y0 = rng.standard_normal(n)
    plan = _plan(D, m, mode)
    for a, b in [(2.5, 0.0), (-1.0, 1.0), (0.75, -0.5)]:
        got = _run(D, m, x, y0, a, b, plan=plan)
        _bound_check(m, x, got, y0, a, b)
        assert np.array_equal(got, _run(D, m, x, y0, a, b, plan=plan, fmt="csr"))
    # beta == 0: y is never read, NaN in y is ignored
    got = _run(D, m, x, np.full(n, np.nan), 1.0, 0.0, plan=plan)
    assert np.isfinite(got).all()


@pytest.mark.parametrize("mode", MODES)
def test_empty_rows_long_rows_ragged(D, cuda_dev, mode):
    """Rows of length 0, 1 and up to 9000 (tiles that exceed a shared-memory
    stage are computed from global memory)."""
    rng = np.random.default_rng(21)
    n = 9000
    lens = rng.integers(0, 6, size=n)
    lens[rng.integers(0, n, size=300)] = 0
    lens[[17, 4000, 8999]] = [9000, 3000, 7000]
    rows = np.repeat(np.arange(n), lens)
    cols = np.concatenate([np.sort(rng.choice(n, size=min(l, n), replace=False)) if l else
                           np.zeros(0, dtype=np.int64) for l in lens])
    keep = np.abs(cols - rows) <= 32767
    rp, col, val = W.from_coo(n, rows[keep], cols[keep], rng.standard_normal(keep.sum()))
    m = Mat(D, cuda_dev, n, n, rp, col, val)
    x = W.uniform_vector(n, rng)
    plan = _plan(D, m, mode)
    got = _run(D, m, x, plan=plan)
    _bound_check(m, x, got)
    assert np.array_equal(got, _run(D, m, x, plan=plan, fmt="csr"))
    assert np.all(got[np.diff(rp) == 0] == 0.0)


@pytest.mark.parametrize("shape", [(5000, 700), (700, 5000), (1, 3000), (3000, 1)])
def test_nonsquare(D, cuda_dev, shape):
    """Remark 3: for nrows != ncols the shifted x is only read in range."""
    nr, nc = shape
    rng = np.random.default_rng(nr + nc)
    rows, cols = [], []
    for r in range(nr):
        k = int(rng.integers(0, 8))
        c = rng.integers(0, nc, size=k)
        rows += [r] * k
        cols += c.tolist()
    rows, cols = np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64)
    keep = np.abs(cols - rows) <= 32767
    rows, cols = rows[keep], cols[keep]
    key = np.unique(rows * nc + cols)
    rp, col, val = W.from_coo(nr, key // nc, key % nc, rng.standard_normal(len(key)))
    m = Mat(D, cuda_dev, nr, nc, rp, col, val)
    x = W.uniform_vector(nc, rng)
    for mode in MODES:
        plan = _plan(D, m, mode)
        got = _run(D, m, x, plan=plan)
        _bound_check(m, x, got)
        assert np.array_equal(got, _run(D, m, x, plan=plan, fmt="csr"))


LOWP = {torch.float32: "f32", torch.bfloat16: "bf16", torch.float8_e4m3fn: "f8e4m3"}


@pytest.mark.parametrize("lowp", list(LOWP))
@pytest.mark.parametrize("mode", MODES)
def test_reduced_precision(D, cuda_dev, lowp, mode):
    rng = np.random.default_rng(31)
    n = 20000
    rp, col, val = W.random_banded(n, 500, rng)
    m = Mat(D, cuda_dev, n, n, rp, col, val, lowp)
    x32 = W.uniform_vector(n, rng).astype(np.float32)
    vq = OS.quantize(val, LOWP[lowp])
    plan = _plan(D, m, mode)
    got = _run(D, m, x32.astype(np.float64), plan=plan)
    _bound_check(m, x32.astype(np.float64), got, u=OS.U32, vals=vq)
    assert np.array_equal(got, _run(D, m, x32.astype(np.float64), plan=plan, fmt="csr"))
    # error against the FP64 matrix, stated per dtype: the value rounding
    # (relative u_v; E4M3 subnormals absolute 2^-10) plus the FP32 sums
    ex64 = OS.spmv_exact(n, rp, m.off, val, x32.astype(np.float64))
    tot = OS.error_bound(n, rp, m.off, vq, x32, u=OS.U32)
    if lowp == torch.float8_e4m3fn:
        tot = tot + OS.UF8 * OS.abs_row_sums(n, rp, m.off, val, x32) + \
            OS.F8_TINY_ABS * OS.abs_row_sums(n, rp, m.off, np.ones_like(val), x32)
    else:
        u_v = OS.U32 if lowp == torch.float32 else OS.UBF16
        tot = tot + u_v * OS.abs_row_sums(n, rp, m.off, val, x32)
    assert np.all(np.abs(got - ex64) <= tot)


def test_config2_full_size_sampled(D, cuda_dev):
    """128^3 7-point Laplacian (n = 2,097,152), natural order, at the size the
    benchmark times: sampled rows against the oracle's Listing 2 order."""
    m_ = 128
    n = m_ ** 3
    rp, col, val = W.laplace3d_7pt(m_)
    m = Mat(D, cuda_dev, n, n, rp, col, val)
    rng = W.rng_for(2, 0)
    x = W.uniform_vector(n, rng)
    plan = D.Plan(m.t_rp, len(col), n, torch.float64, idx=m.t_off)
    got = _run(D, m, x, plan=plan)
    assert np.array_equal(got, _run(D, m, x, plan=plan, fmt="csr"))
    rows = np.unique(np.concatenate([np.arange(0, 300), np.arange(n - 300, n),
                                     rng.integers(0, n, 3000)]))
    ex = OS.spmv_exact(n, rp, m.off, val, x, rows=rows)
    lens = np.diff(rp)[rows].astype(np.float64)
    s = np.array([np.sum(np.abs(val[rp[r]:rp[r + 1]] * x[col[rp[r]:rp[r + 1]]])) for r in rows])
    assert np.all(np.abs(got[rows] - ex) <= 4 * lens * OS.U64 * s)
    # dyadic x: the whole vector is bitwise equal to the oracle
    xd = W.dyadic_vector(n, W.rng_for(2, 2))
    assert np.array_equal(_run(D, m, xd, plan=plan), OS.spmv(n, rp, m.off, val, xd))


def test_empty_matrix_and_zero_rows(D, cuda_dev):
    rp = np.zeros(1001, dtype=np.int32)
    col = np.zeros(0, dtype=np.int32)
    val = np.zeros(0)
    m = Mat(D, cuda_dev, 1000, 1000, rp, col, val)
    x = np.ones(1000)
    for mode in MODES:
        if mode == "none":
            plan = None
        else:
            plan = _plan(D, m, mode)
        assert np.all(_run(D, m, x, plan=plan) == 0.0)
        y0 = np.arange(1000.0)
        assert np.array_equal(_run(D, m, x, y0, 1.0, 2.0, plan=plan), 2.0 * y0)


def test_bounded_wait_selftest(D, cuda_dev):
    """A kernel waiting on a barrier that nothing completes gives up after its
    limit and reports DAMN_ERR_TIMEOUT; the context stays usable."""
    assert D.damn_selftest_wait_timeout(2_000_000) == D.DAMN_ERR_TIMEOUT
    assert D.damn_device_status() == 0
    x = torch.ones(10, dtype=torch.float64, device=cuda_dev)
    assert float(x.sum()) == 10.0


def test_device_status_clean(D, cuda_dev):
    assert D.damn_device_status() == 0


@pytest.mark.parametrize("h", [100, 5000])
def test_heuristic_ragged_rows(D, cuda_dev, h):
    """Random banded rows (lengths LogNormal around 12, row efficiency about
    0.4) get the sorted-rows tiling whatever the band width; within the
    bound and CSR-32 == DA-CSR-16."""
    rng = np.random.default_rng(21)
    n = 20000
    rp, col, val = W.random_banded(n, h, rng)
    m = Mat(D, cuda_dev, n, n, rp, col, val)
    plan = D.Plan(m.t_rp, len(m.col), n, torch.float64, idx=m.t_off)
    d = plan.describe()
    assert 0.3 <= d["row_efficiency"] < 0.85
    assert d["tiling"] == D.DAMN_TILING_SORTED_ROWS, d
    x = W.uniform_vector(n, rng)
    got = _run(D, m, x, plan=plan)
    _bound_check(m, x, got)
    assert np.array_equal(got, _run(D, m, x, plan=plan, fmt="csr"))


@pytest.mark.parametrize("lanes,length", [(1, 7), (2, 20), (4, 50), (8, 100), (16, 200),
                                          (32, 400)])
def test_heuristic_uniform_rows_lanes(D, cuda_dev, lanes, length):
    """Uniform rows get the fewest lanes per row that keep <= 7 (one lane)
    or <= 14 entries per lane."""
    n = 4000
    rows = np.repeat(np.arange(n), length)
    cols = (rows + np.tile(np.arange(length) - length // 2, n)) % n
    rp, col, val = W.from_coo(n, rows, cols, np.random.default_rng(3).standard_normal(len(rows)))
    m = Mat(D, cuda_dev, n, n, rp, col, val)
    plan = D.Plan(m.t_rp, len(col), n, torch.float64, idx=m.t_off)
    want = {1: D.DAMN_TILING_ROWS, 2: D.DAMN_TILING_ROWS_LONG, 4: D.DAMN_TILING_ROWS_LANES4,
            8: D.DAMN_TILING_ROWS_LANES8, 16: D.DAMN_TILING_ROWS_LANES16,
            32: D.DAMN_TILING_ROWS_LANES32}[lanes]
    assert plan.describe()["tiling"] == want
    x = W.uniform_vector(n, np.random.default_rng(4))
    got = _run(D, m, x, plan=plan)
    _bound_check(m, x, got)
    assert np.array_equal(got, _run(D, m, x, plan=plan, fmt="csr"))


@pytest.mark.parametrize("stages", [2, 3, 4, 6])
@pytest.mark.parametrize("tiling", ["band", "sorted", "rows", "rows_x2", "lanes4", "slices"])
def test_ring_depths(D, cuda_dev, tiling, stages):
    """Every ring depth gives the same bits as the automatic depth (the
    summation order does not depend on it)."""
    rng = np.random.default_rng(40 + stages)
    n = 30000
    rp, col, val = W.random_banded(n, 700, rng)
    m = Mat(D, cuda_dev, n, n, rp, col, val)
    x = W.uniform_vector(n, rng)
    plan = _plan(D, m, tiling)
    ref = _run(D, m, x, plan=plan)
    plan.set_stages(stages)
    got = _run(D, m, x, plan=plan)
    assert np.array_equal(got, ref)
    assert plan.describe()["stages_requested"] == stages
    _bound_check(m, x, got)


@pytest.mark.parametrize("h", [300, 2000, 3500, 6000, 30000])
def test_band_ring_and_gather(D, cuda_dev, h):
    """Band and sorted-rows tilings across band widths: x from the ring (narrow bands), partly
    or wholly gathered (bands the 8192-slot ring cannot hold); results within
    the bound, bitwise equal for CSR-32 / DA-CSR-16 and for FP32 values
    between the two formats."""
    rng = np.random.default_rng(h)
    n = 60000
    rp, col, val = W.random_banded(n, h, rng)
    m = Mat(D, cuda_dev, n, n, rp, col, val)
    x = W.uniform_vector(n, rng)
    m32 = Mat(D, cuda_dev, n, n, rp, col, val, torch.float32)
    y0 = rng.standard_normal(n)
    for mode in ("band", "sorted"):
        plan = _plan(D, m, mode)
        got = _run(D, m, x, plan=plan)
        _bound_check(m, x, got)
        assert np.array_equal(got, _run(D, m, x, plan=plan, fmt="csr"))
        got = _run(D, m, x, y0, -0.5, 2.0, plan=plan)
        _bound_check(m, x, got, y0, -0.5, 2.0)
        p32 = _plan(D, m32, mode)
        g32 = _run(D, m32, x.astype(np.float32), plan=p32)
        assert np.array_equal(g32, _run(D, m32, x.astype(np.float32), plan=p32, fmt="csr"))


def test_band_outliers_and_nonsquare(D, cuda_dev):
    """Rows with an entry far from the diagonal (their tiles gather x, the
    ring restarts after them), a tall and a wide matrix, and rows longer
    than a stage (tiles read from global memory)."""
    rng = np.random.default_rng(77)
    n = 50000
    rp, col, val = W.random_banded(n, 200, rng)
    rows = np.repeat(np.arange(n), np.diff(rp))
    far_r = rng.integers(0, n, 40)
    far_c = (far_r + n // 2) % n
    long_r = np.full(5000, 1234)
    long_c = rng.integers(0, 1234 + 30000, 5000)   # offsets within int16
    rr = np.concatenate([rows, far_r, long_r])
    cc = np.concatenate([col, far_c, long_c])
    rp2, col2, val2 = W.from_coo(n, rr, cc, rng.standard_normal(len(rr)))
    assert OD.fit_check(n, n, rp2, col2).fits
    m = Mat(D, cuda_dev, n, n, rp2, col2, val2)
    x = W.uniform_vector(n, rng)
    for mode in ("band", "band_col", "band_gather", "sorted", "sorted_col", "sorted_gather"):
        plan = _plan(D, m, mode)
        got = _run(D, m, x, plan=plan)
        _bound_check(m, x, got)
        assert np.array_equal(got, _run(D, m, x, plan=plan, fmt="csr"))
    for nr, nc in ((30000, 9000), (9000, 30000)):
        rpn, coln, valn = W.random_banded_rect(nr, nc, 400, rng)
        mn = Mat(D, cuda_dev, nr, nc, rpn, coln, valn)
        xn = W.uniform_vector(nc, rng)
        for mode in ("band", "sorted"):
            plan = _plan(D, mn, mode)
            got = _run(D, mn, xn, plan=plan)
            _bound_check(mn, xn, got)
            assert np.array_equal(got, _run(D, mn, xn, plan=plan, fmt="csr"))


@pytest.mark.parametrize("h", [300, 30000])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32, torch.bfloat16])
def test_band_without_ring_same_bits(D, cuda_dev, h, dt):
    """The band tiling with its x ring and without it (x staging off: every
    tile gathers x from global memory, the ring's shared memory left to L1)
    gives the same bits -- the ring only changes where x comes from -- for
    both index formats, with and without a requested ring depth."""
    rng = np.random.default_rng(500 + h)
    n = 40000
    rp, col, val = W.random_banded(n, h, rng)
    m = Mat(D, cuda_dev, n, n, rp, col, val, dt)
    x = W.uniform_vector(n, rng)
    plan = _plan(D, m, "band")
    ring = _run(D, m, x, plan=plan)
    ring_csr = _run(D, m, x, plan=plan, fmt="csr")
    plan.set_x_staging(False)
    assert plan.describe()["x_staging"] == 0
    assert np.array_equal(_run(D, m, x, plan=plan), ring)
    assert np.array_equal(_run(D, m, x, plan=plan, fmt="csr"), ring_csr)
    plan.set_stages(8)
    assert np.array_equal(_run(D, m, x, plan=plan), ring)
    assert np.array_equal(ring, ring_csr)
    assert D.damn_device_status() == D.DAMN_OK
