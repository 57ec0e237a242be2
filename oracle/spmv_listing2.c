/*
 * Plain C restatement of Listing 2 (Section 4.1): y <- alpha*A*x + beta*y for
 * CSR with 32-bit column indices and DA-CSR with 16-bit diagonal offsets,
 * FP64 values.  Rows are split across OpenMP threads with a static schedule,
 * the paper's own parallelisation (Section 4.1).
 *
 * TEST INFRASTRUCTURE ONLY: this is the oracle's timed CPU baseline.  It is
 * compiled with -ffp-contract=off so that each product and sum is rounded
 * separately, matching oracle/spmv.py bit for bit; beta == 0 leaves y
 * unread (BLAS convention).
 */
#include <stdint.h>
#include <omp.h>

int oracle_max_threads(void) { return omp_get_max_threads(); }

void oracle_spmv_csr32_f64(int32_t nrows, const int32_t *rowptr, const int32_t *colids,
                           const double *values, const double *x, double *y,
                           double alpha, double beta, int nthreads) {
#pragma omp parallel for schedule(static) num_threads(nthreads)
  for (int32_t row = 0; row < nrows; ++row) {
    double accumulator = 0.0;
    for (int32_t i = rowptr[row]; i < rowptr[row + 1]; ++i) {
      accumulator += values[i] * x[colids[i]];
    }
    y[row] = (beta == 0.0) ? alpha * accumulator : alpha * accumulator + beta * y[row];
  }
}

void oracle_spmv_dacsr16_f64(int32_t nrows, const int32_t *rowptr, const int16_t *colids,
                             const double *values, const double *x, double *y,
                             double alpha, double beta, int nthreads) {
#pragma omp parallel for schedule(static) num_threads(nthreads)
  for (int32_t row = 0; row < nrows; ++row) {
    double accumulator = 0.0;
    const double *xshift = x + row; /* only dereferenced at in-range columns */
    for (int32_t i = rowptr[row]; i < rowptr[row + 1]; ++i) {
      accumulator += values[i] * xshift[colids[i]];
    }
    y[row] = (beta == 0.0) ? alpha * accumulator : alpha * accumulator + beta * y[row];
  }
}
