"""Seeded synthetic inputs for the DA-CSR SpMV workloads.

This module is shared by the CPU oracle (``oracle/``), the tests and
``bench.py``.  It only *builds inputs*: sparsity patterns, values and vectors
drawn from a fixed-seed PCG64 stream.  It holds none of the method's arithmetic
(no index translation, no bandwidth computation, no products), so the oracle
and the CUDA path stay independent of each other.

The paper evaluates on SuiteSparse matrices (Section 3), which are not
available here; the generators below are stand-ins with the structure the
paper relies on: low bandwidth (possibly only after reordering), tens of
entries per row, and a total traffic that ranges from in-cache to far beyond
cache (Section 4.2).

Every matrix is returned in CSR form as ``(rowptr, col, val)`` with
``rowptr`` int32[nrows+1], ``col`` int32[nnz] (column indices ascending inside
each row) and ``val`` float64[nnz].

Workloads (sizes as used by the tests and the benchmark):

* ``laplace2d_5pt(64)``: 2-D 5-point Laplacian on a 64x64 grid, natural order.
* ``laplace3d_7pt(128)``: 3-D 7-point Laplacian on a 128^3 grid, natural
  order, or with a seeded random relabelling of the grid vertices
  (``scrambled=True``), which breaks the 16-bit fit.
* ``random_banded(n, h, seed)``: random banded rows with log-normal row
  lengths (median 12, sigma 0.5, clipped to 1..200), diagonal always present.
* ``stencil27(160)``: SPD 3-D 27-point stencil (diagonal 26.5, others -1).
* ``batch_banded(512, seed)``: 512 independent random banded matrices with
  log-normal sizes in [1e3, 2e5], 5..40 entries per row, half-bandwidth
  drawn from 16..4096.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20230712


def seed_for(config_index: int, variant: int = 0) -> int:
    """Seed of the PCG64 stream for workload ``config_index`` (1-based)."""
    return BASE_SEED + 1000 * int(config_index) + int(variant)


def rng_for(config_index: int, variant: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config_index, variant)))


# ----------------------------------------------------------------------------
# Vectors
# ----------------------------------------------------------------------------

def uniform_vector(n: int, rng: np.random.Generator, dtype=np.float64) -> np.ndarray:
    """x ~ U[-1, 1)."""
    return rng.uniform(-1.0, 1.0, size=int(n)).astype(dtype)


def dyadic_vector(n: int, rng: np.random.Generator, bits: int = 20) -> np.ndarray:
    """x uniform on the grid {k * 2^-bits} inside [-1, 1].

    Used with small-integer matrix values so that every partial sum of a row
    product is exactly representable (any summation order gives the same
    bits)."""
    k = rng.integers(-(1 << bits), (1 << bits) + 1, size=int(n))
    return np.ldexp(k.astype(np.float64), -bits)


def uniform_block(n: int, k: int, rng: np.random.Generator, dtype=np.float64) -> np.ndarray:
    """Row-major n x k block of right-hand sides, U[-1, 1)."""
    return rng.uniform(-1.0, 1.0, size=(int(n), int(k))).astype(dtype)


# ----------------------------------------------------------------------------
# Grid stencils
# ----------------------------------------------------------------------------

def _assemble_rows(label_of_vertex: np.ndarray, nbr_vertex: np.ndarray, nbr_valid: np.ndarray,
                   nbr_value: np.ndarray, n: int):
    """Assemble CSR rows from per-vertex neighbour lists.

    ``nbr_vertex`` [nvert, S] lists the stencil neighbours of each grid vertex
    (``nbr_valid`` masks those outside the grid) and ``nbr_value`` [S] the
    matrix value of each stencil slot.  Row ``label_of_vertex[v]`` receives
    column ``label_of_vertex[nbr]`` for every valid neighbour; columns are
    sorted ascending inside each row."""
    nvert, S = nbr_vertex.shape
    counts = nbr_valid.sum(axis=1).astype(np.int64)
    row_of_vertex = label_of_vertex
    # rows are ordered by label: count per row
    row_counts = np.empty(n, dtype=np.int64)
    row_counts[row_of_vertex] = counts
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(row_counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    # vertex-major scatter, then per-row sort by column label
    cols_lab = np.where(nbr_valid, label_of_vertex[np.where(nbr_valid, nbr_vertex, 0)], np.iinfo(np.int64).max)
    order = np.argsort(cols_lab, axis=1, kind="stable")
    cols_sorted = np.take_along_axis(cols_lab, order, axis=1)
    vals_sorted = np.broadcast_to(nbr_value, (nvert, S))
    vals_sorted = np.take_along_axis(vals_sorted, order, axis=1)
    # the valid entries are the first counts[v] of each sorted row
    slot = np.arange(S)[None, :]
    keep = slot < counts[:, None]
    starts = rowptr[row_of_vertex]  # [nvert]
    dest = (starts[:, None] + slot)[keep]
    col[dest] = cols_sorted[keep].astype(np.int32)
    val[dest] = vals_sorted[keep]
    return rowptr.astype(np.int32), col, val


def _grid_stencil(dims, offsets, values, labels=None):
    dims = tuple(int(d) for d in dims)
    nvert = int(np.prod(dims))
    coords = np.indices(dims).reshape(len(dims), -1).T  # [nvert, D], C order
    offs = np.asarray(offsets, dtype=np.int64)  # [S, D]
    nb = coords[:, None, :] + offs[None, :, :]  # [nvert, S, D]
    valid = np.all((nb >= 0) & (nb < np.asarray(dims)[None, None, :]), axis=2)
    strides = np.array([int(np.prod(dims[i + 1:])) for i in range(len(dims))], dtype=np.int64)
    nbr = (nb * strides[None, None, :]).sum(axis=2)
    if labels is None:
        labels = np.arange(nvert, dtype=np.int64)
    return _assemble_rows(np.asarray(labels, dtype=np.int64), nbr, valid,
                          np.asarray(values, dtype=np.float64), nvert)


def laplace2d_5pt(m: int = 64):
    """2-D 5-point Laplacian on an m x m grid, natural (row-major) order:
    4 on the diagonal, -1 for the four grid neighbours."""
    offs = [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    vals = [-1.0, -1.0, 4.0, -1.0, -1.0]
    return _grid_stencil((m, m), offs, vals)


def laplace2d_5pt_rect(mx: int, my: int):
    """2-D 5-point Laplacian on a grid of my lines of mx points, natural
    (row-major) order: half-bandwidth mx."""
    offs = [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    vals = [-1.0, -1.0, 4.0, -1.0, -1.0]
    return _grid_stencil((my, mx), offs, vals)


def _chunked_stencil(m: int, offsets, values, labels=None, chunk_planes: int = 8):
    """3-D stencil assembled plane block by plane block (bounded memory)."""
    if labels is None:
        return _grid_stencil_natural_3d(m, offsets, values)
    return _grid_stencil((m, m, m), offsets, values, labels)


def _grid_stencil_natural_3d(m: int, offsets, values):
    """Natural-order 3-D stencil assembled in bounded-memory slabs.

    In natural order the rows are the vertices themselves, so each slab of
    x-planes can be assembled independently and concatenated."""
    n = m ** 3
    offs = np.asarray(offsets, dtype=np.int64)
    vals = np.asarray(values, dtype=np.float64)
    order = np.lexsort((offs[:, 2], offs[:, 1], offs[:, 0]))  # ascending linear offset
    offs, vals = offs[order], vals[order]
    lin = offs[:, 0] * m * m + offs[:, 1] * m + offs[:, 2]
    counts_all = []
    cols_all = []
    vals_all = []
    slab = max(1, (1 << 22) // (m * m))
    for x0 in range(0, m, slab):
        x1 = min(m, x0 + slab)
        c = np.indices((x1 - x0, m, m)).reshape(3, -1).T
        c[:, 0] += x0
        nb = c[:, None, :] + offs[None, :, :]
        valid = np.all((nb >= 0) & (nb < m), axis=2)
        v = (c[:, 0] * m * m + c[:, 1] * m + c[:, 2])
        colm = v[:, None] + lin[None, :]
        counts_all.append(valid.sum(axis=1))
        cols_all.append(colm[valid].astype(np.int32))
        vals_all.append(np.broadcast_to(vals, valid.shape)[valid])
    counts = np.concatenate(counts_all)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr.astype(np.int32), np.concatenate(cols_all), np.concatenate(vals_all)


def laplace3d_7pt(m: int = 128, scrambled: bool = False, rng: np.random.Generator | None = None):
    """3-D 7-point Laplacian on an m^3 grid: 6 on the diagonal, -1 for the six
    grid neighbours.

    ``scrambled=False`` numbers the vertices in natural (row-major) order.
    ``scrambled=True`` numbers them by a seeded random bijection drawn from
    ``rng`` (``rng.permutation``); this is the same grid graph under another
    vertex numbering, whose bandwidth is close to n."""
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    vals = [-1.0, -1.0, -1.0, 6.0, -1.0, -1.0, -1.0]
    if not scrambled:
        return _grid_stencil_natural_3d(m, offs, vals)
    if rng is None:
        rng = rng_for(2, 1)
    labels = rng.permutation(m ** 3).astype(np.int64)
    return _grid_stencil((m, m, m), offs, vals, labels)


def stencil27(m: int = 160, diag: float = 26.5, off: float = -1.0):
    """SPD 3-D 27-point stencil on an m^3 grid, natural order: ``diag`` on the
    diagonal, ``off`` for the 26 neighbours in the 3x3x3 box."""
    offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    vals = [diag if o == (0, 0, 0) else off for o in offs]
    return _grid_stencil_natural_3d(m, offs, vals)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on uint64 counters."""
    z = (z + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    return z ^ (z >> np.uint64(31))


def perturb_symmetric(n: int, rowptr, col, val, sigma: float = 0.01, seed: int | None = None,
                      chunk: int = 1 << 24):
    """Adds N(0, sigma^2) to every off-diagonal entry, the same value to
    (i, j) and (j, i): the normal is drawn (Box-Muller) from a counter-based
    hash of the unordered pair, so no pairing pass is needed.  Returns new
    values; A stays symmetric."""
    if seed is None:
        seed = seed_for(4, 7)
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    out = np.array(val, dtype=np.float64, copy=True)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    for a in range(0, len(col), chunk):
        r, c = rows[a:a + chunk], col[a:a + chunk]
        key = (np.minimum(r, c) * np.int64(n) + np.maximum(r, c)).astype(np.uint64)
        h1 = _splitmix64(key ^ s)
        h2 = _splitmix64(h1)
        u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53   # (0, 1]
        u2 = (h2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        out[a:a + chunk] += np.where(r != c, sigma * g, 0.0)
    return out


# ----------------------------------------------------------------------------
# Random banded matrices
# ----------------------------------------------------------------------------

def _banded_rows(n: int, h_lo, h_hi, k: np.ndarray, rng: np.random.Generator,
                 row0: int = 0):
    """Column sets for rows row0..row0+len(k)-1 of an n x n banded matrix.

    Row r draws k[r]-1 columns uniformly (with replacement) from its window
    [max(0, r-h), min(n-1, r+h)], adds the diagonal, removes duplicates and
    sorts.  Returns (counts, cols)."""
    nr = len(k)
    r = np.arange(row0, row0 + nr, dtype=np.int64)
    lo = np.maximum(0, r - h_lo)
    hi = np.minimum(n - 1, r + h_hi)
    width = hi - lo + 1
    extra = np.maximum(k - 1, 0)
    rr = np.repeat(np.arange(nr, dtype=np.int64), extra)
    draw = rng.integers(0, width[rr])
    cols = np.concatenate([lo[rr] + draw, r])
    rows = np.concatenate([rr, np.arange(nr, dtype=np.int64)])
    key = rows * n + cols
    key.sort()
    keep = np.ones(len(key), dtype=bool)
    np.not_equal(key[1:], key[:-1], out=keep[1:])
    key = key[keep]                      # sorted, duplicates removed
    rows_u = key // n
    cols_u = key - rows_u * n
    counts = np.bincount(rows_u, minlength=nr)
    return counts, cols_u.astype(np.int32)


def random_banded(n: int, h: int, rng: np.random.Generator, median: float = 12.0,
                  sigma: float = 0.5, kmin: int = 1, kmax: int = 200, chunk_rows: int = 1 << 20):
    """Seeded random banded n x n matrix.

    Row lengths k_r = clip(round(LogNormal(ln median, sigma)), kmin, kmax);
    columns as in ``_banded_rows``; values N(0, 1)."""
    n = int(n)
    k = np.clip(np.rint(rng.lognormal(np.log(median), sigma, size=n)), kmin, kmax).astype(np.int64)
    counts_all, cols_all = [], []
    for r0 in range(0, n, chunk_rows):
        c, cols = _banded_rows(n, h, h, k[r0:r0 + chunk_rows], rng, r0)
        counts_all.append(c)
        cols_all.append(cols)
    counts = np.concatenate(counts_all)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    assert rowptr[-1] < 2 ** 31
    col = np.concatenate(cols_all)
    val = rng.standard_normal(len(col))
    return rowptr.astype(np.int32), col, val


def random_banded_rect(nrows: int, ncols: int, h: int, rng: np.random.Generator,
                       median: float = 12.0, sigma: float = 0.5):
    """Seeded random banded nrows x ncols matrix: row r draws its entries
    (count as in ``random_banded``) uniformly from the columns within h of r
    that exist, [max(0, r - h), min(ncols - 1, r + h)]; rows whose window is
    empty (r - h >= ncols) stay empty.  Values N(0, 1)."""
    k = np.clip(np.rint(rng.lognormal(np.log(median), sigma, size=nrows)), 1, 200).astype(np.int64)
    r = np.arange(nrows, dtype=np.int64)
    lo = np.maximum(0, r - h)
    hi = np.minimum(ncols - 1, r + h)
    ok = hi >= lo
    k = np.where(ok, k, 0)
    rr = np.repeat(r, k)
    cols = lo[rr] + rng.integers(0, (hi - lo + 1)[rr])
    key = np.unique(rr * ncols + cols)
    rows_u, cols_u = key // ncols, key % ncols
    return from_coo(nrows, rows_u, cols_u, rng.standard_normal(len(key)))


def batch_banded(count: int = 512, seed: int | None = None, n_median: float = 14142.0,
                 n_sigma: float = 1.0, n_min: int = 1000, n_max: int = 200000,
                 k_min: int = 5, k_max: int = 40, h_min: int = 16, h_max: int = 4096):
    """``count`` independent random banded square matrices.

    n = clip(round(LogNormal(ln n_median, n_sigma)), n_min, n_max), row
    lengths uniform in k_min..k_max (then deduplicated), one half-bandwidth per
    matrix uniform in h_min..h_max, values N(0, 1), diagonal always present.
    Returns a list of (n, rowptr, col, val)."""
    if seed is None:
        seed = seed_for(5)
    top = np.random.Generator(np.random.PCG64(seed))
    ns = np.clip(np.rint(top.lognormal(np.log(n_median), n_sigma, size=count)), n_min, n_max).astype(np.int64)
    hs = top.integers(h_min, h_max + 1, size=count)
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64([seed, i]))
        n = int(ns[i])
        k = rng.integers(k_min, k_max + 1, size=n).astype(np.int64)
        counts, col = _banded_rows(n, int(hs[i]), int(hs[i]), k, rng)
        rowptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(counts, out=rowptr[1:])
        val = rng.standard_normal(len(col))
        out.append((n, rowptr.astype(np.int32), col, val))
    return out


# ----------------------------------------------------------------------------
# Small hand-made patterns used by the tests
# ----------------------------------------------------------------------------

def example1_pattern():
    """The 4x4 sample matrix of Fig. 1 / Example 1 (entries (0,0), (1,2),
    (2,1), (2,3), (3,3)); the paper draws its values as colours, so values
    are chosen here as 1..5."""
    rowptr = np.array([0, 1, 2, 4, 5], dtype=np.int32)
    col = np.array([0, 2, 1, 3, 3], dtype=np.int32)
    val = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    return rowptr, col, val


def from_coo(n_rows: int, rows, cols, vals=None):
    """CSR arrays from coordinate lists, rows grouped and columns sorted
    (duplicates kept in input order)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    if vals is None:
        vals = np.ones(len(rows))
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], np.asarray(vals, dtype=np.float64)[order]
    counts = np.bincount(rows, minlength=n_rows)
    rowptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr.astype(np.int32), cols.astype(np.int32), vals


def block_stencil3d(m: int, b: int, rng: np.random.Generator | None = None):
    """Block sparse matrix with the pattern of the 3-D 7-point stencil on an
    m^3 grid (natural order) and dense b x b blocks (b unknowns per grid
    point, as in 3-D elasticity): block values N(0, 1), plus 2 b on the
    diagonal of each diagonal block.  Returns (nbr, browptr, bcol,
    bval[nblk, b, b])."""
    if rng is None:
        rng = rng_for(6, b)
    rp, col, _ = laplace3d_7pt(m)
    nbr = m ** 3
    nblk = len(col)
    bval = rng.standard_normal((nblk, b, b))
    rows = np.repeat(np.arange(nbr, dtype=np.int64), np.diff(rp.astype(np.int64)))
    diag = rows == col
    bval[diag] += 2.0 * b * np.eye(b)[None, :, :]
    return nbr, rp, col, bval
