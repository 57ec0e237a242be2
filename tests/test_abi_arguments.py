"""Argument checks of the C ABI, on the CPU: every entry point rejects bad
sizes, NULL pointers, unsupported dtypes or formats, misaligned pointers and
too-small workspaces with the status code its header comment documents,
names itself in damn_last_error(), and does so before any device work (the
pointers passed here are never dereferenced; no GPU is needed)."""
import ctypes

import pytest

N = None
A16 = 0x10000          # a 16-byte aligned address the checks must not touch
A8 = 0x10008           # 8-byte aligned only


@pytest.fixture(scope="module")
def D():
    from paper_2307_06305_gb300 import build as B
    B.build()
    from paper_2307_06305_gb300 import damn
    return damn


def _cases(D):
    F = D._fn
    fi = lambda: ctypes.byref(D.damn_fit_info())
    i64 = lambda: ctypes.byref(D.I64(0))
    out = lambda: ctypes.byref(ctypes.c_void_p())
    cg = lambda: ctypes.byref(D.damn_cg_result())
    bad, uns = D.DAMN_ERR_INVALID_ARG, D.DAMN_ERR_UNSUPPORTED
    return [
        # SpMV (CSR-32, DA-CSR-16, DA-CSR-8)
        ("damn_spmv_dacsr16", bad, "bad sizes",
         lambda: F("damn_spmv_dacsr16")(-1, 4, 0, N, N, N, 0, N, N, 1.0, 0.0, N, N)),
        ("damn_spmv_dacsr16", bad, "NULL",
         lambda: F("damn_spmv_dacsr16")(4, 4, 4, N, A16, A16, 0, A16, A16, 1.0, 0.0, N, N)),
        ("damn_spmv_dacsr16", bad, "NULL",
         lambda: F("damn_spmv_dacsr16")(4, 4, 4, A16, A16, N, 0, A16, A16, 1.0, 0.0, N, N)),
        ("damn_spmv_dacsr16", bad, "dtype",
         lambda: F("damn_spmv_dacsr16")(4, 4, 4, A16, A16, A16, 7, A16, A16, 1.0, 0.0, N, N)),
        ("damn_spmv_dacsr16", bad, "aligned",
         lambda: F("damn_spmv_dacsr16")(4, 4, 4, A16, A16, A16, 0, A8, A16, 1.0, 0.0, N, N)),
        ("damn_spmv_dacsr16", bad, "aligned",
         lambda: F("damn_spmv_dacsr16")(4, 4, 4, A16, A16, A8, 0, A16, A16, 1.0, 0.0, N, N)),
        ("damn_spmv_csr32", bad, "bad sizes",
         lambda: F("damn_spmv_csr32")(4, 4, 1 << 31, A16, A16, A16, 0, A16, A16, 1.0, 0.0, N, N)),
        ("damn_spmv_dacsr8", bad, "bad sizes",
         lambda: F("damn_spmv_dacsr8")(4, -4, 4, A16, A16, A16, 0, A16, A16, 1.0, 0.0, N, N)),
        # conversion and checks
        ("damn_csr_to_dacsr", bad, "NULL",
         lambda: F("damn_csr_to_dacsr")(4, 4, 4, A16, A16, A16, N, A16, 1 << 20, N)),
        ("damn_csr_to_dacsr", bad, "workspace",
         lambda: F("damn_csr_to_dacsr")(4, 4, 4, A16, A16, A16, fi(), A16, 0, N)),
        ("damn_csr_to_dacsr8", bad, "bad sizes",
         lambda: F("damn_csr_to_dacsr8")(4, 4, -1, A16, A16, A16, fi(), A16, 1 << 20, N)),
        ("damn_csr_to_dacsr_noalloc", bad, "static scratch",
         lambda: F("damn_csr_to_dacsr_noalloc")(D.DAMN_NOALLOC_MAX_ROWS + 1, 4, 0, A16, A16, A16,
                                                fi(), N)),
        ("damn_validate_csr", bad, "bad sizes",
         lambda: F("damn_validate_csr")(-1, 4, 0, A16, A16, i64(), i64(), A16, 1 << 20, N)),
        ("damn_validate_dacsr", bad, "bad sizes",
         lambda: F("damn_validate_dacsr")(-1, 4, 0, A16, A16, 16, i64(), i64(), A16, 1 << 20, N)),
        ("damn_validate_dacsr", bad, "off_bits",
         lambda: F("damn_validate_dacsr")(4, 4, 4, A16, A16, 32, i64(), i64(), A16, 1 << 20, N)),
        ("damn_validate_dacsr", bad, "workspace",
         lambda: F("damn_validate_dacsr")(4, 4, 4, A16, A16, 16, i64(), i64(), A16, 0, N)),
        ("damn_cast_values", uns, "dtype",
         lambda: F("damn_cast_values")(10, A16, 0, A16, 0, N)),
        ("damn_cast_values", bad, "n < 0",
         lambda: F("damn_cast_values")(-1, A16, 0, A16, 1, N)),
        # plans
        ("damn_plan_create", bad, "bad",
         lambda: F("damn_plan_create")(-1, 4, 0, N, 1, N, 0, N, out())),
        ("damn_plan_create", bad, "format",
         lambda: F("damn_plan_create")(4, 4, 4, A16, 9, A16, 0, N, out())),
        ("damn_plan_create", bad, "NULL",
         lambda: F("damn_plan_create")(4, 4, 4, A16, 1, A16, 0, N, N)),
        ("damn_plan_describe", bad, "NULL",
         lambda: F("damn_plan_describe")(N, ctypes.byref(D.damn_plan_desc()))),
        ("damn_plan_set_tiling", bad, "NULL",
         lambda: F("damn_plan_set_tiling")(N, 1)),
        ("damn_plan_autotune", bad, "NULL",
         lambda: F("damn_plan_autotune")(N, 1, A16, A16, A16, A16, N)),
        # COO / BSR
        ("damn_spmv_dacoo16", bad, "bad sizes",
         lambda: F("damn_spmv_dacoo16")(-1, 4, 0, N, N, N, 0, N, N, 1.0, 0.0, N, 0, N)),
        ("damn_spmv_coo32", bad, "workspace",
         lambda: F("damn_spmv_coo32")(4, 4, 4, A16, A16, A16, 0, A16, A16, 1.0, 0.0, A16, 0, N)),
        ("damn_spmv_bsr32", uns, "block size",
         lambda: F("damn_spmv_bsr32")(4, 4, 4, 5, A16, A16, A16, 0, A16, A16, 1.0, 0.0, N)),
        ("damn_spmv_dabsr16", bad, "bad sizes",
         lambda: F("damn_spmv_dabsr16")(-1, 4, 4, 2, A16, A16, A16, 0, A16, A16, 1.0, 0.0, N)),
        # RCM / permutation
        ("damn_rcm_permute", bad, "bad sizes",
         lambda: F("damn_rcm_permute")(-1, 0, N, N, N, 0, N, N, N, N,
                                       ctypes.byref(D.damn_bw_info()), N, 0, N)),
        ("damn_permute_sym", bad, "workspace",
         lambda: F("damn_permute_sym")(4, 4, A16, A16, N, 0, A16, A16, A16, N, A16, 0, N)),
        # solvers
        ("damn_cg", bad, "bad sizes",
         lambda: F("damn_cg")(-1, 0, N, N, N, N, N, 1e-10, 10, N, cg(), N, 0, N)),
        ("damn_cg", bad, "workspace",
         lambda: F("damn_cg")(4, 4, A16, A16, A16, A16, A16, 1e-10, 10, N, cg(), A16, 0, N)),
        ("damn_cg_ir", bad, "low_dtype",
         lambda: F("damn_cg_ir")(4, 4, A16, A16, A16, A16, 0, A16, A16, 1e-10, 1e-3, 10, 10, N, N,
                                 cg(), A16, 1 << 24, N)),
        # SpMM and batches
        ("damn_spmm_dacsr16", bad, "k must be",
         lambda: F("damn_spmm_dacsr16")(4, 4, 4, A16, A16, A16, 0, 0, A16, A16, N)),
        ("damn_spmm_dacsr16", bad, "bad arguments",  # entries but no column of X
         lambda: F("damn_spmm_dacsr16")(4, 0, 4, A16, A16, A16, 0, 1, A16, A16, N)),
        ("damn_spmm_dacsr16", bad, "bad arguments",  # no headroom below INT_MAX
         lambda: F("damn_spmm_dacsr16")(4, 4, 2**31 - 10, A16, A16, A16, 0, 1, A16, A16, N)),
        ("damn_batch_plan_create", bad, "count",
         lambda: F("damn_batch_plan_create")(-1, N, 1, 0, 0, N, out())),
        ("damn_batch_plan_create", bad, "k must be",
         lambda: F("damn_batch_plan_create")(0, N, 0, 0, 0, N, out())),
        ("damn_spmm_dacsr16_batched", bad, "NULL",
         lambda: F("damn_spmm_dacsr16_batched")(N, N)),
        ("damn_batch_graph_launch", bad, "NULL",
         lambda: F("damn_batch_graph_launch")(N, N)),
        ("damn_batch_plan_set_shape", bad, "NULL",
         lambda: F("damn_batch_plan_set_shape")(N, 1, 64, 1, 128, N)),
        # diagnostics
        ("damn_selftest_wait_timeout", bad, "timeout_ns",
         lambda: F("damn_selftest_wait_timeout")(5, N)),
        ("damn_device_status", bad, "NULL",
         lambda: F("damn_device_status")(N, 0, N)),
    ]


def test_rejections_before_device_work(D):
    seen = set()
    for name, want, words, call in _cases(D):
        rc = call()
        msg = D.last_error()
        assert rc == want, (name, rc, msg)
        assert words in msg, (name, msg)
        if "block size" not in words:
            assert msg.startswith(name), (name, msg)
        seen.add(name)
    # every compute entry point of the header is covered
    assert {"damn_spmv_csr32", "damn_spmv_dacsr16", "damn_spmv_dacsr8", "damn_csr_to_dacsr",
            "damn_csr_to_dacsr8", "damn_csr_to_dacsr_noalloc", "damn_cg", "damn_cg_ir",
            "damn_spmm_dacsr16", "damn_batch_plan_create", "damn_permute_sym",
            "damn_rcm_permute", "damn_plan_create"} <= seen


def test_destroy_null_is_a_no_op(D):
    assert D._fn("damn_plan_destroy")(N) == D.DAMN_OK
    assert D._fn("damn_batch_plan_destroy")(N) == D.DAMN_OK
