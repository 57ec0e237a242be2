// SpMV kernels for csr32 indices and FP8 E4M3 values (see spmv_launch.cuh).
#include "spmv_launch.cuh"

DAMN_SPMV_INSTANCE(spmv_launch_csr32_f8, damn::f8e4m3, int32_t)
