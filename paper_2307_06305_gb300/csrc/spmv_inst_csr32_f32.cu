// SpMV kernels for csr32 indices and f32 values (see spmv_launch.cuh).
#include "spmv_launch.cuh"

DAMN_SPMV_INSTANCE(spmv_launch_csr32_f32, float, int32_t)
