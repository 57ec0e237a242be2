// Internal interface of the SpMV engine, shared by the SpMV entry points, the
// CG solvers and the plan code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/damn.h"

namespace damn {

// One SpMV launch: y = alpha * A x + beta * y0, optionally also a per-CTA
// partial sum of dot_w[r] * y[r] (or y[r]^2 when dot_self) written to
// dot_partials[blockIdx.x] in FP64.
struct SpmvCall {
  int32_t nrows = 0, ncols = 0;
  int64_t nnz = 0;
  const int32_t *rowptr = nullptr;
  const void *idx = nullptr;    // int32 col (CSR-32) or int16 off (DA-CSR-16)
  int fmt = DAMN_FMT_DACSR16;
  const void *val = nullptr;
  int dtype = DAMN_F64;
  const void *x = nullptr;
  const void *y0 = nullptr;     // beta term input (may alias y)
  void *y = nullptr;
  double alpha = 1.0, beta = 0.0;
  const void *dot_w = nullptr;
  int dot_self = 0;
  double *dot_partials = nullptr;
};

// Launches the SpMV kernel selected by `plan` (NULL: fixed row tiles with
// balanced slices).  *grid_out (optional) receives the number of CTAs, i.e.
// of dot partials written.
int spmv_launch(const SpmvCall &c, const damn_plan *plan, cudaStream_t s, int *grid_out);

// Upper bound of the number of CTAs (dot partials) spmv_launch may use.
int spmv_max_grid();

// DAMN_OK when plan is NULL or was built for this matrix: same sizes and
// dtype, the same rowptr array, and the same index array when fmt is the
// plan's own format (another format's copy of the same matrix is allowed).
// Otherwise DAMN_ERR_INVALID_ARG with a message naming fn.
int plan_check(const char *fn, const damn_plan *plan, int fmt, int32_t nrows, int32_t ncols,
               int64_t nnz, const int32_t *rowptr, const void *idx, int dtype);

}  // namespace damn
