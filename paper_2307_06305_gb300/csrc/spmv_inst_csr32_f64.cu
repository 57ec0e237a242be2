// SpMV kernels for csr32 indices and f64 values (see spmv_launch.cuh).
#include "spmv_launch.cuh"

DAMN_SPMV_INSTANCE(spmv_launch_csr32_f64, double, int32_t)
