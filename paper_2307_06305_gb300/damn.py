"""Thin Python binding of the DA-CSR CUDA library (``include/damn.h``).

Argument marshalling only: every function takes torch tensors that live on
the current CUDA device, passes their device pointers and the current CUDA
stream to the C entry point of the same name, and raises ``DamnError`` on a
non-zero status.  All arithmetic runs in the library's kernels; there is no
CPU fallback, and importing this module fails loudly when the compiled library
is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdamn.so")

DAMN_OK = 0
DAMN_ERR_INVALID_ARG = -1
DAMN_ERR_NOFIT = -2
DAMN_ERR_CUDA = -3
DAMN_ERR_NOT_CONVERGED = -4
DAMN_ERR_TIMEOUT = -5
DAMN_ERR_UNSUPPORTED = -6

DAMN_F64, DAMN_F32, DAMN_BF16 = 0, 1, 2
DAMN_FMT_CSR32, DAMN_FMT_DACSR16, DAMN_FMT_DACSR8 = 0, 1, 2
DAMN_TILING_SLICES, DAMN_TILING_ROWS, DAMN_TILING_ROWS_LONG, DAMN_TILING_BAND = 0, 1, 2, 3
DAMN_TILING_ROWS_LANES4, DAMN_TILING_ROWS_LANES8 = 4, 5
DAMN_TILING_ROWS_LANES16, DAMN_TILING_ROWS_LANES32 = 6, 7
DAMN_TILING_SORTED_ROWS, DAMN_TILING_ROWS_X2 = 8, 9

DAMN_F8E4M3 = 3
_DTYPE_CODE = {torch.float64: DAMN_F64, torch.float32: DAMN_F32, torch.bfloat16: DAMN_BF16,
               torch.float8_e4m3fn: DAMN_F8E4M3}
_VEC_DTYPE = {DAMN_F64: torch.float64, DAMN_F32: torch.float32, DAMN_BF16: torch.float32,
              DAMN_F8E4M3: torch.float32}


class DamnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


if not os.path.exists(LIB_PATH):
    raise ImportError(f"DA-CSR CUDA library not built: {LIB_PATH} is missing "
                      "(run paper_2307_06305_gb300/build.py or __graft_entry__.build())")

_lib = ctypes.CDLL(LIB_PATH)

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
F64 = ctypes.c_double
SZ = ctypes.c_size_t


class damn_fit_info(ctypes.Structure):
    _fields_ = [("min_off", I32), ("max_off", I32), ("w", I64), ("n_fit", I64), ("n_bad", I64),
                ("fits", I32), ("reserved", I32)]


class damn_bw_info(ctypes.Structure):
    _fields_ = [("w_before", I64), ("w_after", I64)]


class damn_plan_desc(ctypes.Structure):
    _fields_ = [("mode", I32), ("tile_items", I32), ("ntiles", I32), ("grid", I32),
                ("stages", I32), ("threads", I32), ("row_efficiency", F64), ("max_row", I32),
                ("dtype", I32), ("tiling", I32), ("x_staged_tiles", I32),
                ("stages_requested", I32), ("x_staging", I32)]


class damn_cg_result(ctypes.Structure):
    _fields_ = [("iterations", I32), ("outer", I32), ("converged", I32), ("reserved", I32),
                ("relres", F64), ("true_relres", F64)]


class damn_mat_desc(ctypes.Structure):
    _fields_ = [("nrows", I32), ("ncols", I32), ("nnz", I64), ("rowptr", P), ("off", P),
                ("val", P), ("X", P), ("Y", P)]


class damn_batch_desc(ctypes.Structure):
    _fields_ = [("count", I32), ("k", I32), ("dtype", I32), ("ntiles", I32), ("grid", I32),
                ("threads", I32), ("tile_items", I32), ("graph_ready", I32),
                ("entry_lanes", I32), ("streamed", I32), ("tune_ms", F64)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("damn_last_error", ctypes.c_char_p, [])
_sig("damn_version", ctypes.c_int, [])
_sig("damn_device_status", ctypes.c_int, [ctypes.POINTER(I32), ctypes.c_int, P])
_sig("damn_selftest_wait_timeout", ctypes.c_int, [I64, P])
_sig("damn_csr_to_dacsr_workspace_size", SZ, [])
_sig("damn_csr_to_dacsr", ctypes.c_int,
     [I32, I32, I64, P, P, P, ctypes.POINTER(damn_fit_info), P, SZ, P])
_sig("damn_csr_to_dacsr8", ctypes.c_int,
     [I32, I32, I64, P, P, P, ctypes.POINTER(damn_fit_info), P, SZ, P])
_sig("damn_csr_to_dacsr_noalloc", ctypes.c_int,
     [I32, I32, I64, P, P, P, ctypes.POINTER(damn_fit_info), P])
_sig("damn_validate_csr_workspace_size", SZ, [])
_sig("damn_validate_dacsr", ctypes.c_int,
     [I32, I32, I64, P, P, I32, ctypes.POINTER(I64), ctypes.POINTER(I64), P, SZ, P])
_sig("damn_validate_csr", ctypes.c_int,
     [I32, I32, I64, P, P, ctypes.POINTER(I64), ctypes.POINTER(I64), P, SZ, P])
_sig("damn_cast_values", ctypes.c_int, [I64, P, ctypes.c_int, P, ctypes.c_int, P])
_sig("damn_plan_create", ctypes.c_int,
     [I32, I32, I64, P, ctypes.c_int, P, ctypes.c_int, P, ctypes.POINTER(P)])
_sig("damn_plan_autotune", ctypes.c_int, [P, ctypes.c_int, P, P, P, P, P])
_sig("damn_plan_describe", ctypes.c_int, [P, ctypes.POINTER(damn_plan_desc)])
_sig("damn_plan_set_tiling", ctypes.c_int, [P, ctypes.c_int])
_sig("damn_plan_set_stages", ctypes.c_int, [P, I32])
_sig("damn_plan_set_x_staging", ctypes.c_int, [P, I32])
_sig("damn_plan_destroy", ctypes.c_int, [P])
_sig("damn_spmv_csr32", ctypes.c_int,
     [I32, I32, I64, P, P, P, ctypes.c_int, P, P, F64, F64, P, P])
_sig("damn_spmv_dacsr16", ctypes.c_int,
     [I32, I32, I64, P, P, P, ctypes.c_int, P, P, F64, F64, P, P])
_sig("damn_spmv_dacsr8", ctypes.c_int,
     [I32, I32, I64, P, P, P, ctypes.c_int, P, P, F64, F64, P, P])
_sig("damn_coo_workspace_size", SZ, [I64, ctypes.c_int])
for _n in ("damn_spmv_coo32", "damn_spmv_dacoo16"):
    _sig(_n, ctypes.c_int, [I32, I32, I64, P, P, P, ctypes.c_int, P, P, F64, F64, P, SZ, P])
for _n in ("damn_spmv_bsr32", "damn_spmv_dabsr16", "damn_spmv_dabsr8"):
    _sig(_n, ctypes.c_int, [I32, I32, I64, I32, P, P, P, ctypes.c_int, P, P, F64, F64, P])

_OPTIONAL = {}


def _opt(name, res, args):
    """Declares a required symbol (a missing one fails the import)."""
    _OPTIONAL[name] = _sig(name, res, args)


_opt("damn_rcm_order", ctypes.c_int, [I32, I64, P, P, P, ctypes.POINTER(I64), ctypes.POINTER(I64)])
_opt("damn_permute_sym_workspace_size", SZ, [I32])
_opt("damn_permute_sym", ctypes.c_int, [I32, I64, P, P, P, ctypes.c_int, P, P, P, P, P, SZ, P])
_opt("damn_rcm_permute", ctypes.c_int,
     [I32, I64, P, P, P, ctypes.c_int, P, P, P, P, ctypes.POINTER(damn_bw_info), P, SZ, P])
_opt("damn_cg_workspace_size", SZ, [I32])
_opt("damn_cg", ctypes.c_int,
     [I32, I64, P, P, P, P, P, F64, I32, P, ctypes.POINTER(damn_cg_result), P, SZ, P])
_opt("damn_cg_ir_workspace_size", SZ, [I32])
_opt("damn_cg_ir", ctypes.c_int,
     [I32, I64, P, P, P, P, ctypes.c_int, P, P, F64, F64, I32, I32, P, P,
      ctypes.POINTER(damn_cg_result), P, SZ, P])
_opt("damn_spmm_dacsr16", ctypes.c_int, [I32, I32, I64, P, P, P, ctypes.c_int, I32, P, P, P])
_opt("damn_batch_plan_create", ctypes.c_int,
     [I32, ctypes.POINTER(damn_mat_desc), I32, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(P)])
_opt("damn_batch_plan_describe", ctypes.c_int, [P, ctypes.POINTER(damn_batch_desc)])
_opt("damn_batch_plan_set_shape", ctypes.c_int, [P, I32, I32, I32, I32, P])
_opt("damn_batch_plan_destroy", ctypes.c_int, [P])
_opt("damn_spmm_dacsr16_batched", ctypes.c_int, [P, P])
_opt("damn_batch_graph_launch", ctypes.c_int, [P, P])


def _fn(name):
    if name in _OPTIONAL:
        return _OPTIONAL[name]
    return getattr(_lib, name)


def last_error() -> str:
    return _lib.damn_last_error().decode(errors="replace")


def _check(rc: int, what: str, allow=()):
    if rc != DAMN_OK and rc not in allow:
        raise DamnError(rc, f"{what}: {last_error()}")
    return rc


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


def damn_version() -> int:
    return int(_lib.damn_version())


def loaded_library_path() -> str:
    return LIB_PATH


# ----------------------------------------------------------------------------
# diagnostics
# ----------------------------------------------------------------------------

def damn_device_status(reset: bool = False, stream=None) -> int:
    v = I32(0)
    _check(_lib.damn_device_status(ctypes.byref(v), int(reset), _stream(stream)), "damn_device_status")
    return int(v.value)


def damn_selftest_wait_timeout(timeout_ns: int, stream=None) -> int:
    """Returns the library status (DAMN_ERR_TIMEOUT when the bounded wait gave up)."""
    return int(_lib.damn_selftest_wait_timeout(int(timeout_ns), _stream(stream)))


# ----------------------------------------------------------------------------
# a1: conversion and fit check
# ----------------------------------------------------------------------------

@dataclass
class FitInfo:
    min_off: int
    max_off: int
    w: int
    n_fit: int
    n_bad: int
    fits: bool


def damn_csr_to_dacsr(rowptr: torch.Tensor, col: torch.Tensor, ncols: int, off_out=None,
                      stream=None, raise_on_nofit: bool = False):
    """Returns (off int16 tensor, FitInfo).  off is unspecified when not fits."""
    nrows = rowptr.numel() - 1
    nnz = col.numel()
    if off_out is None:
        off_out = torch.empty(nnz, dtype=torch.int16, device=col.device)
    ws = _workspace(_lib.damn_csr_to_dacsr_workspace_size(), col.device)
    info = damn_fit_info()
    rc = _lib.damn_csr_to_dacsr(nrows, int(ncols), nnz, _ptr(rowptr), _ptr(col), _ptr(off_out),
                                ctypes.byref(info), _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "damn_csr_to_dacsr", allow=() if raise_on_nofit else (DAMN_ERR_NOFIT,))
    return off_out, FitInfo(info.min_off, info.max_off, info.w, info.n_fit, info.n_bad,
                            bool(info.fits))


def damn_csr_to_dacsr8(rowptr: torch.Tensor, col: torch.Tensor, ncols: int, off_out=None,
                       stream=None, raise_on_nofit: bool = False):
    """CSR -> DA-CSR-8: returns (off int8 tensor, FitInfo with the int8 fit)."""
    nrows = rowptr.numel() - 1
    nnz = col.numel()
    if off_out is None:
        off_out = torch.empty(nnz, dtype=torch.int8, device=col.device)
    ws = _workspace(_lib.damn_csr_to_dacsr_workspace_size(), col.device)
    info = damn_fit_info()
    rc = _lib.damn_csr_to_dacsr8(nrows, int(ncols), nnz, _ptr(rowptr), _ptr(col), _ptr(off_out),
                                 ctypes.byref(info), _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "damn_csr_to_dacsr8", allow=() if raise_on_nofit else (DAMN_ERR_NOFIT,))
    return off_out, FitInfo(info.min_off, info.max_off, info.w, info.n_fit, info.n_bad,
                            bool(info.fits))


DAMN_NOALLOC_MAX_ROWS = 1048576


def damn_csr_to_dacsr_noalloc(rowptr: torch.Tensor, col: torch.Tensor, ncols: int,
                              off_out: torch.Tensor, stream=None, raise_on_nofit: bool = False):
    """CSR -> DA-CSR-16 without any device allocation, for callers that
    cannot allocate (their framework owns all device memory, or cudaMalloc's
    device-wide synchronisation is not acceptable on their path).  The
    caller provides ``off_out``; the library's static scratch limits the
    matrix to DAMN_NOALLOC_MAX_ROWS rows.  Returns (off_out, FitInfo)."""
    nrows = rowptr.numel() - 1
    info = damn_fit_info()
    rc = _lib.damn_csr_to_dacsr_noalloc(nrows, int(ncols), col.numel(), _ptr(rowptr), _ptr(col),
                                        _ptr(off_out), ctypes.byref(info), _stream(stream))
    _check(rc, "damn_csr_to_dacsr_noalloc", allow=() if raise_on_nofit else (DAMN_ERR_NOFIT,))
    return off_out, FitInfo(info.min_off, info.max_off, info.w, info.n_fit, info.n_bad,
                            bool(info.fits))


def damn_validate_csr(rowptr, col, ncols: int, stream=None):
    nrows = rowptr.numel() - 1
    ws = _workspace(_lib.damn_validate_csr_workspace_size(), rowptr.device)
    br, bc = I64(0), I64(0)
    rc = _lib.damn_validate_csr(nrows, int(ncols), col.numel(), _ptr(rowptr), _ptr(col),
                                ctypes.byref(br), ctypes.byref(bc), _ptr(ws), ws.numel(),
                                _stream(stream))
    _check(rc, "damn_validate_csr", allow=(DAMN_ERR_INVALID_ARG,))
    return int(br.value), int(bc.value)


def damn_validate_dacsr(rowptr, off, ncols: int, stream=None):
    """(bad row pointers, entries with r + off outside [0, ncols)) of a
    DA-CSR-16 (int16 off) or DA-CSR-8 (int8 off) matrix."""
    nrows = rowptr.numel() - 1
    ws = _workspace(_lib.damn_validate_csr_workspace_size(), rowptr.device)
    br, bc = I64(0), I64(0)
    bits = 8 if off.dtype == torch.int8 else 16
    rc = _lib.damn_validate_dacsr(nrows, int(ncols), off.numel(), _ptr(rowptr), _ptr(off), bits,
                                  ctypes.byref(br), ctypes.byref(bc), _ptr(ws), ws.numel(),
                                  _stream(stream))
    _check(rc, "damn_validate_dacsr", allow=(DAMN_ERR_INVALID_ARG,))
    return int(br.value), int(bc.value)


def damn_cast_values(src: torch.Tensor, dst_dtype: torch.dtype, stream=None) -> torch.Tensor:
    dst = torch.empty(src.numel(), dtype=dst_dtype, device=src.device)
    rc = _lib.damn_cast_values(src.numel(), _ptr(src), _DTYPE_CODE[src.dtype], _ptr(dst),
                               _DTYPE_CODE[dst_dtype], _stream(stream))
    _check(rc, "damn_cast_values")
    return dst


# ----------------------------------------------------------------------------
# SpMV and plans
# ----------------------------------------------------------------------------

class Plan:
    """Owns a damn_plan (tiling, compute mode, x windows) for one matrix and
    one value dtype.  ``idx`` is the column array (int32 col for CSR-32,
    int16 / int8 off for DA-CSR-16 / DA-CSR-8; None: no x windows).  Keep rowptr and idx alive
    while the plan is used."""

    def __init__(self, rowptr: torch.Tensor, nnz: int, ncols: int, dtype: torch.dtype, idx=None,
                 stream=None):
        self.handle = P()
        self.rowptr = rowptr
        self.idx = idx
        self.dtype_code = _DTYPE_CODE[dtype]
        fmt = DAMN_FMT_CSR32
        if idx is not None and idx.dtype == torch.int16:
            fmt = DAMN_FMT_DACSR16
        elif idx is not None and idx.dtype == torch.int8:
            fmt = DAMN_FMT_DACSR8
        rc = _lib.damn_plan_create(rowptr.numel() - 1, int(ncols), int(nnz), _ptr(rowptr), fmt,
                                   _ptr(idx), self.dtype_code, _stream(stream),
                                   ctypes.byref(self.handle))
        _check(rc, "damn_plan_create")

    def autotune(self, fmt: int, idx, val, x, y, stream=None):
        rc = _lib.damn_plan_autotune(self.handle, int(fmt), _ptr(idx), _ptr(val), _ptr(x), _ptr(y),
                                     _stream(stream))
        _check(rc, "damn_plan_autotune")
        return self

    def set_tiling(self, tiling: int):
        _check(_lib.damn_plan_set_tiling(self.handle, int(tiling)), "damn_plan_set_tiling")
        return self

    def set_x_staging(self, on: bool):
        """Rows tilings: stage x windows in shared memory (True) or read x
        from global memory (False)."""
        _check(_lib.damn_plan_set_x_staging(self.handle, int(bool(on))), "damn_plan_set_x_staging")
        return self

    def set_stages(self, stages: int):
        """Ring depth of the plan's launches (0: automatic, else 2..8)."""
        _check(_lib.damn_plan_set_stages(self.handle, int(stages)), "damn_plan_set_stages")
        return self

    def describe(self) -> dict:
        d = damn_plan_desc()
        _check(_lib.damn_plan_describe(self.handle, ctypes.byref(d)), "damn_plan_describe")
        return {k: getattr(d, k) for k, _ in damn_plan_desc._fields_}

    def close(self):
        if self.handle:
            _lib.damn_plan_destroy(self.handle)
            self.handle = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def damn_plan_create(rowptr, nnz, ncols, dtype, idx=None, stream=None) -> Plan:
    return Plan(rowptr, nnz, ncols, dtype, idx, stream)


def _plan_handle(plan):
    return None if plan is None else plan.handle


def damn_spmv_csr32(rowptr, col, val, x, y, alpha=1.0, beta=0.0, plan=None, ncols=None, stream=None):
    nrows = rowptr.numel() - 1
    ncols = x.numel() if ncols is None else ncols
    rc = _lib.damn_spmv_csr32(nrows, int(ncols), col.numel(), _ptr(rowptr), _ptr(col), _ptr(val),
                              _DTYPE_CODE[val.dtype], _ptr(x), _ptr(y), float(alpha), float(beta),
                              _plan_handle(plan), _stream(stream))
    _check(rc, "damn_spmv_csr32")
    return y


def damn_spmv_dacsr16(rowptr, off, val, x, y, alpha=1.0, beta=0.0, plan=None, ncols=None,
                      stream=None):
    nrows = rowptr.numel() - 1
    ncols = x.numel() if ncols is None else ncols
    rc = _lib.damn_spmv_dacsr16(nrows, int(ncols), off.numel(), _ptr(rowptr), _ptr(off), _ptr(val),
                                _DTYPE_CODE[val.dtype], _ptr(x), _ptr(y), float(alpha),
                                float(beta), _plan_handle(plan), _stream(stream))
    _check(rc, "damn_spmv_dacsr16")
    return y


def damn_spmv_dacsr8(rowptr, off, val, x, y, alpha=1.0, beta=0.0, plan=None, ncols=None,
                     stream=None):
    nrows = rowptr.numel() - 1
    ncols = x.numel() if ncols is None else ncols
    rc = _lib.damn_spmv_dacsr8(nrows, int(ncols), off.numel(), _ptr(rowptr), _ptr(off), _ptr(val),
                               _DTYPE_CODE[val.dtype], _ptr(x), _ptr(y), float(alpha),
                               float(beta), _plan_handle(plan), _stream(stream))
    _check(rc, "damn_spmv_dacsr8")
    return y


def _bsr_call(name, browptr, bidx, val, b, x, y, alpha, beta, nbc, stream):
    nbr = browptr.numel() - 1
    nbc = (x.numel() // b) if nbc is None else nbc
    rc = getattr(_lib, name)(nbr, int(nbc), bidx.numel(), int(b), _ptr(browptr), _ptr(bidx),
                             _ptr(val), _DTYPE_CODE[val.dtype], _ptr(x), _ptr(y), float(alpha),
                             float(beta), _stream(stream))
    _check(rc, name)
    return y


def damn_spmv_bsr32(browptr, bcol, val, b, x, y, alpha=1.0, beta=0.0, nbc=None, stream=None):
    """Block CSR SpMV; val is [nblk * b * b] (blocks row-major)."""
    return _bsr_call("damn_spmv_bsr32", browptr, bcol, val, b, x, y, alpha, beta, nbc, stream)


def damn_spmv_dabsr16(browptr, boff, val, b, x, y, alpha=1.0, beta=0.0, nbc=None, stream=None):
    """DA-BSR SpMV with int16 block offsets (from damn_csr_to_dacsr on the block pattern)."""
    return _bsr_call("damn_spmv_dabsr16", browptr, boff, val, b, x, y, alpha, beta, nbc, stream)


def damn_spmv_dabsr8(browptr, boff, val, b, x, y, alpha=1.0, beta=0.0, nbc=None, stream=None):
    """DA-BSR SpMV with int8 block offsets (from damn_csr_to_dacsr8 on the block pattern)."""
    return _bsr_call("damn_spmv_dabsr8", browptr, boff, val, b, x, y, alpha, beta, nbc, stream)


def _coo_call(name, nrows, row, idx, val, x, y, alpha, beta, ncols, stream, workspace):
    ncols = x.numel() if ncols is None else ncols
    dt = _DTYPE_CODE[val.dtype]
    ws = workspace if workspace is not None else \
        _workspace(_lib.damn_coo_workspace_size(idx.numel(), dt), y.device)
    rc = getattr(_lib, name)(int(nrows), int(ncols), idx.numel(), _ptr(row), _ptr(idx), _ptr(val),
                             dt, _ptr(x), _ptr(y), float(alpha), float(beta), _ptr(ws), ws.numel(),
                             _stream(stream))
    _check(rc, name)
    return y


def damn_spmv_coo32(nrows, row, col, val, x, y, alpha=1.0, beta=0.0, ncols=None, stream=None,
                    workspace=None):
    """COO SpMV, entries sorted by row."""
    return _coo_call("damn_spmv_coo32", nrows, row, col, val, x, y, alpha, beta, ncols, stream,
                     workspace)


def damn_spmv_dacoo16(nrows, row, off, val, x, y, alpha=1.0, beta=0.0, ncols=None, stream=None,
                      workspace=None):
    """DA-COO SpMV: int16 offsets c - r instead of columns, entries sorted by row."""
    return _coo_call("damn_spmv_dacoo16", nrows, row, off, val, x, y, alpha, beta, ncols, stream,
                     workspace)


# ----------------------------------------------------------------------------
# a6: CG and CG-IR
# ----------------------------------------------------------------------------

def _cg_result(res, rc):
    return {"iterations": int(res.iterations), "outer": int(res.outer),
            "converged": bool(res.converged), "relres": float(res.relres),
            "true_relres": float(res.true_relres), "status": int(rc)}


def damn_cg(rowptr, off, val, b, x, rtol=1e-10, max_iter=1000, plan=None, stream=None,
            workspace=None):
    """FP64 CG on a DA-CSR-16 SPD matrix; x holds x0 on entry and the solution
    on exit.  Returns a dict (iterations, converged, relres, true_relres)."""
    n = rowptr.numel() - 1
    need = _fn("damn_cg_workspace_size")(n)
    ws = workspace if workspace is not None else _workspace(need, b.device)
    res = damn_cg_result()
    rc = _fn("damn_cg")(n, off.numel(), _ptr(rowptr), _ptr(off), _ptr(val), _ptr(b), _ptr(x),
                        float(rtol), int(max_iter), _plan_handle(plan), ctypes.byref(res), _ptr(ws),
                        ws.numel(), _stream(stream))
    _check(rc, "damn_cg", allow=(DAMN_ERR_NOT_CONVERGED,))
    return _cg_result(res, rc)


def damn_cg_ir(rowptr, off, val, val_low, b, x, rtol=1e-10, inner_rtol=1e-3, max_inner=100,
               max_outer=50, plan64=None, plan_low=None, stream=None, workspace=None):
    """Mixed-precision refinement: FP64 residual / update, inner CG with
    val_low (float32 or bfloat16 values), FP32 vectors and FP64 dots."""
    n = rowptr.numel() - 1
    need = _fn("damn_cg_ir_workspace_size")(n)
    ws = workspace if workspace is not None else _workspace(need, b.device)
    res = damn_cg_result()
    rc = _fn("damn_cg_ir")(n, off.numel(), _ptr(rowptr), _ptr(off), _ptr(val), _ptr(val_low),
                           _DTYPE_CODE[val_low.dtype], _ptr(b), _ptr(x), float(rtol),
                           float(inner_rtol), int(max_inner), int(max_outer), _plan_handle(plan64),
                           _plan_handle(plan_low), ctypes.byref(res), _ptr(ws), ws.numel(),
                           _stream(stream))
    _check(rc, "damn_cg_ir", allow=(DAMN_ERR_NOT_CONVERGED,))
    return _cg_result(res, rc)


# ----------------------------------------------------------------------------
# a7: multi-RHS SpMM, single and batched
# ----------------------------------------------------------------------------

def damn_spmm_dacsr16(rowptr, off, val, X, Y, stream=None):
    """Y = A X for one DA-CSR-16 matrix; X [ncols, k], Y [nrows, k] row-major."""
    nrows = rowptr.numel() - 1
    k = X.shape[1]
    rc = _fn("damn_spmm_dacsr16")(nrows, X.shape[0], off.numel(), _ptr(rowptr), _ptr(off),
                                  _ptr(val), _DTYPE_CODE[val.dtype], k, _ptr(X), _ptr(Y),
                                  _stream(stream))
    _check(rc, "damn_spmm_dacsr16")
    return Y


class BatchPlan:
    """A batch of independent products Y_m = A_m X_m (DA-CSR-16) run by one
    persistent launch (and its captured CUDA graph).  ``mats`` is a list of
    (rowptr, off, val, X, Y) tensors that must stay alive with the plan."""

    def __init__(self, mats, k: int, dtype: torch.dtype, autotune: bool = True, stream=None):
        self.mats = mats
        arr = (damn_mat_desc * max(1, len(mats)))()
        for i, (rp, off, val, X, Y) in enumerate(mats):
            arr[i] = damn_mat_desc(rp.numel() - 1, X.shape[0], off.numel(), rp.data_ptr(),
                                   off.data_ptr(), val.data_ptr(), X.data_ptr(), Y.data_ptr())
        self.handle = P()
        rc = _fn("damn_batch_plan_create")(len(mats), arr, int(k), _DTYPE_CODE[dtype],
                                           int(bool(autotune)), _stream(stream),
                                           ctypes.byref(self.handle))
        _check(rc, "damn_batch_plan_create")

    def launch(self, stream=None):
        _check(_fn("damn_spmm_dacsr16_batched")(self.handle, _stream(stream)),
               "damn_spmm_dacsr16_batched")

    def graph_launch(self, stream=None):
        _check(_fn("damn_batch_graph_launch")(self.handle, _stream(stream)),
               "damn_batch_graph_launch")

    def set_shape(self, streamed: bool, rows_per_item: int, entry_lanes: int = 1,
                  threads: int = 256, stream=None):
        """Pins the launch shape (streamed rows or fixed passes, entry_lanes
        lanes per row) and captures the graph again."""
        _check(_fn("damn_batch_plan_set_shape")(self.handle, int(bool(streamed)), int(rows_per_item),
                                                int(entry_lanes), int(threads), _stream(stream)),
               "damn_batch_plan_set_shape")

    def describe(self) -> dict:
        d = damn_batch_desc()
        _check(_fn("damn_batch_plan_describe")(self.handle, ctypes.byref(d)),
               "damn_batch_plan_describe")
        return {k: getattr(d, k) for k, _ in damn_batch_desc._fields_}

    def close(self):
        if self.handle:
            _fn("damn_batch_plan_destroy")(self.handle)
            self.handle = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# a2: RCM ordering and the symmetric permutation
# ----------------------------------------------------------------------------

def damn_rcm_order(h_rowptr, h_col):
    """Host RCM ordering of a square pattern given as host (numpy int32)
    arrays; returns (perm new->old int32, w_before, w_after)."""
    import numpy as np
    rp = np.ascontiguousarray(h_rowptr, dtype=np.int32)
    col = np.ascontiguousarray(h_col, dtype=np.int32)
    n = rp.size - 1
    perm = np.empty(max(n, 1), dtype=np.int32)
    wb, wa = I64(0), I64(0)
    rc = _fn("damn_rcm_order")(n, col.size, rp.ctypes.data, col.ctypes.data if col.size else None,
                               perm.ctypes.data, ctypes.byref(wb), ctypes.byref(wa))
    _check(rc, "damn_rcm_order")
    return perm[:n], int(wb.value), int(wa.value)


def _perm_outputs(n, nnz, val, device):
    rp_out = torch.empty(n + 1, dtype=torch.int32, device=device)
    col_out = torch.empty(max(nnz, 1), dtype=torch.int32, device=device)[:nnz]
    val_out = None if val is None else torch.empty(max(nnz, 1), dtype=val.dtype, device=device)[:nnz]
    return rp_out, col_out, val_out


def damn_permute_sym(rowptr, col, val, perm, stream=None):
    """B = P A P^T on the device; returns (rowptr_out, col_out, val_out)."""
    n = rowptr.numel() - 1
    nnz = col.numel()
    rp_out, col_out, val_out = _perm_outputs(n, nnz, val, rowptr.device)
    ws = _workspace(_fn("damn_permute_sym_workspace_size")(n), rowptr.device)
    dt = _DTYPE_CODE[val.dtype] if val is not None else DAMN_F64
    rc = _fn("damn_permute_sym")(n, nnz, _ptr(rowptr), _ptr(col), _ptr(val), dt, _ptr(perm),
                                 _ptr(rp_out), _ptr(col_out), _ptr(val_out), _ptr(ws), ws.numel(),
                                 _stream(stream))
    _check(rc, "damn_permute_sym")
    return rp_out, col_out, val_out


def damn_rcm_permute(rowptr, col, val, stream=None):
    """RCM ordering + P A P^T; returns (perm, rowptr_out, col_out, val_out,
    {"w_before", "w_after"}).  Synchronises."""
    n = rowptr.numel() - 1
    nnz = col.numel()
    rp_out, col_out, val_out = _perm_outputs(n, nnz, val, rowptr.device)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=rowptr.device)[:n]
    ws = _workspace(_fn("damn_permute_sym_workspace_size")(n), rowptr.device)
    info = damn_bw_info()
    dt = _DTYPE_CODE[val.dtype] if val is not None else DAMN_F64
    rc = _fn("damn_rcm_permute")(n, nnz, _ptr(rowptr), _ptr(col), _ptr(val), dt, _ptr(perm),
                                 _ptr(rp_out), _ptr(col_out), _ptr(val_out), ctypes.byref(info),
                                 _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "damn_rcm_permute")
    return perm, rp_out, col_out, val_out, {"w_before": info.w_before, "w_after": info.w_after}
