/*
 * CPU baseline of the oracle: y = alpha A x (+ beta y) for FP64 matrices
 * stored as CSR with 32-bit column indices and as DA-CSR with 16-bit
 * diagonal offsets.  What it computes is Section 4's SpMV (Listing 2): every
 * row is summed from zero over its entries in stored order, product by
 * product, and the sum is then scaled by alpha, with beta y added when beta
 * is non-zero (beta == 0 leaves y unread, the BLAS convention).  The rows
 * are divided among OpenMP threads in equal contiguous blocks, as in the
 * paper's parallel runs (Section 4.1).
 *
 * TEST INFRASTRUCTURE ONLY: this is the oracle's timed CPU baseline.  Built
 * with -ffp-contract=off, so every product and every sum is rounded on its
 * own and the result equals oracle/spmv.py bit for bit.
 */
#include <stdint.h>
#include <omp.h>

int oracle_max_threads(void) { return omp_get_max_threads(); }

/* Row r's result from its sum s. */
static inline double finish_row(double s, double alpha, double beta, const double *y, int32_t r) {
  if (beta == 0.0) return alpha * s;
  return alpha * s + beta * y[r];
}

/* CSR-32: entry k of row r multiplies x[col[k]]. */
void oracle_spmv_csr32_f64(int32_t nrows, const int32_t *rowptr, const int32_t *col,
                           const double *val, const double *x, double *y,
                           double alpha, double beta, int nthreads) {
#pragma omp parallel for schedule(static) num_threads(nthreads)
  for (int32_t r = 0; r < nrows; ++r) {
    const int32_t end = rowptr[r + 1];
    double s = 0.0;
    for (int32_t k = rowptr[r]; k != end; ++k) s = s + val[k] * x[col[k]];
    y[r] = finish_row(s, alpha, beta, y, r);
  }
}

/* DA-CSR-16: entry k of row r multiplies x[r + off[k]] (Section 2: the
 * stored index is the column minus the row). */
void oracle_spmv_dacsr16_f64(int32_t nrows, const int32_t *rowptr, const int16_t *off,
                             const double *val, const double *x, double *y,
                             double alpha, double beta, int nthreads) {
#pragma omp parallel for schedule(static) num_threads(nthreads)
  for (int32_t r = 0; r < nrows; ++r) {
    const int32_t end = rowptr[r + 1];
    double s = 0.0;
    for (int32_t k = rowptr[r]; k != end; ++k) s = s + val[k] * x[(int64_t)r + off[k]];
    y[r] = finish_row(s, alpha, beta, y, r);
  }
}
